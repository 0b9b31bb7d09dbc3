// Launch counting and per-kernel-class timing (CUDA events on the launching stream) with device-side
// accumulation of the algorithmic flops/bytes of the launches (ranks live on the device).
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace tpcg {

std::atomic<long long> g_launches{0};
thread_local long long t_launches = 0;

namespace {
struct EvPair {
    cudaEvent_t a, b;
    int kind;
};
std::mutex g_mu;
bool g_on = false;
double* g_dev = nullptr;                // PK_COUNT * 2 doubles: flops, bytes
std::vector<EvPair> g_pairs;            // recorded (start, stop) pairs
std::vector<cudaEvent_t> g_free;        // recycled events
// index of the open pair per kind, per host thread (concurrent solves open and close pairs independently)
thread_local std::vector<int> g_open(PK_COUNT, -1);
long long g_gen = 0;                    // bumped by every reset: a thread's open pairs of an older generation are void
thread_local long long t_gen = 0;
void sync_gen() {
    if (t_gen != g_gen) {
        for (int k = 0; k < PK_COUNT; ++k) g_open[k] = -1;
        t_gen = g_gen;
    }
}
long long g_count[PK_COUNT] = {0};

cudaEvent_t get_event() {
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

bool prof_on() { return g_on; }
double* prof_dev() { return g_on ? g_dev : nullptr; }

void prof_begin(int kind, cudaStream_t st) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    sync_gen();
    EvPair p{get_event(), get_event(), kind};
    cudaEventRecord(p.a, st);
    g_open[kind] = (int)g_pairs.size();
    g_pairs.push_back(p);
}

void prof_end(int kind, cudaStream_t st) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    sync_gen();
    int i = g_open[kind];
    if (i < 0 || i >= (int)g_pairs.size()) return;
    cudaEventRecord(g_pairs[i].b, st);
    g_open[kind] = -1;
    g_count[kind]++;
}

}  // namespace tpcg

using namespace tpcg;

extern "C" long long tpcg_launch_count(void) { return g_launches.load(); }

extern "C" int tpcg_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (on && !g_dev) {
        if (cudaMalloc(&g_dev, PK_COUNT * 2 * sizeof(double)) != cudaSuccess) {
            g_dev = nullptr;
            set_error("tpcg_profile_enable: cudaMalloc failed");
            return TPCG_E_NOMEM;
        }
        if (sync_zero(g_dev, PK_COUNT * 2 * sizeof(double)) != TPCG_OK) return TPCG_E_CUDA;
    }
    g_on = on != 0;
    return TPCG_OK;
}

extern "C" int tpcg_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaDeviceSynchronize();
    for (auto& p : g_pairs) {
        g_free.push_back(p.a);
        g_free.push_back(p.b);
    }
    g_pairs.clear();
    ++g_gen;
    for (int k = 0; k < PK_COUNT; ++k) {
        g_open[k] = -1;
        g_count[k] = 0;
    }
    if (g_dev && sync_zero(g_dev, PK_COUNT * 2 * sizeof(double)) != TPCG_OK) return TPCG_E_CUDA;
    return TPCG_OK;
}

extern "C" int tpcg_profile_get(int kind, double* ms_total, long long* count, double* flops, double* bytes) {
    if (kind < 0 || kind >= PK_COUNT) return TPCG_E_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaDeviceSynchronize();
    double ms = 0;
    for (auto& p : g_pairs) {
        if (p.kind != kind) continue;
        float t = 0;
        if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) ms += t;
    }
    if (ms_total) *ms_total = ms;
    if (count) *count = g_count[kind];
    double h[2] = {0, 0};
    if (g_dev) cudaMemcpy(h, g_dev + 2 * kind, sizeof(h), cudaMemcpyDeviceToHost);
    if (flops) *flops = h[0];
    if (bytes) *bytes = h[1];
    return TPCG_OK;
}

namespace tpcg {
static std::atomic<int> g_gemm_ctas_per_sm{2};
int gemm_ctas_per_sm() { return g_gemm_ctas_per_sm.load(std::memory_order_relaxed); }
static std::atomic<int> g_expsum_kind{1};
int expsum_kind() { return g_expsum_kind.load(std::memory_order_relaxed); }
static std::atomic<int> g_eig_kind{1};
int eig_kind() { return g_eig_kind.load(std::memory_order_relaxed); }
static std::atomic<int> g_dst_kind{1};
int dst_kind() { return g_dst_kind.load(std::memory_order_relaxed); }
static std::atomic<int> g_tc_kind{0};
int tc_kind() { return g_tc_kind.load(std::memory_order_relaxed); }
static std::atomic<int> g_rr_kind{1};
int rr_kind() { return g_rr_kind.load(std::memory_order_relaxed); }
static std::atomic<int> g_gemm_kind{2};
int gemm_kind() { return g_gemm_kind.load(std::memory_order_relaxed); }
static std::atomic<int> g_gram_min_k{0};
int gram_min_k() { return g_gram_min_k.load(std::memory_order_relaxed); }
static std::atomic<int> g_round_rule{-1};
int round_rule() { return g_round_rule.load(std::memory_order_relaxed); }
static std::atomic<int> g_resolved{1};
int resolved_kind() { return g_resolved.load(std::memory_order_relaxed); }
}  // namespace tpcg

extern "C" int tpcg_set_option(int key, long long value) {
    if (key == TPCG_OPT_GEMM_CTAS_PER_SM && value >= 0 && value <= 64) {
        tpcg::g_gemm_ctas_per_sm.store((int)value);
        return TPCG_OK;
    }
    if (key == TPCG_OPT_EXPSUM_BEST && (value == 0 || value == 1)) {
        tpcg::g_expsum_kind.store((int)value);
        return TPCG_OK;
    }
    if (key == TPCG_OPT_EIG && (value == 0 || value == 1)) {
        tpcg::g_eig_kind.store((int)value);
        return TPCG_OK;
    }
    if (key == TPCG_OPT_DST && (value == 0 || value == 1)) {
        tpcg::g_dst_kind.store((int)value);
        return TPCG_OK;
    }
    if (key == TPCG_OPT_TC && (value == 0 || value == 1)) {
        tpcg::g_tc_kind.store((int)value);
        return TPCG_OK;
    }
    if (key == TPCG_OPT_RR && (value == 0 || value == 1)) {
        tpcg::g_rr_kind.store((int)value);
        return TPCG_OK;
    }
    if (key == TPCG_OPT_GEMM_KIND && value >= 0 && value <= 2) {
        tpcg::g_gemm_kind.store((int)value);
        return TPCG_OK;
    }
    if (key == TPCG_OPT_RESOLVED && (value == 0 || value == 1)) {
        tpcg::g_resolved.store((int)value);
        return TPCG_OK;
    }
    if (key == TPCG_OPT_ROUND_RULE && value >= -1 && value <= 2) {
        tpcg::g_round_rule.store((int)value);
        return TPCG_OK;
    }
    if (key == TPCG_OPT_GRAM_MIN_K && value >= 0 && value <= (1 << 24)) {
        tpcg::g_gram_min_k.store((int)value);
        return TPCG_OK;
    }
    tpcg::set_error("tpcg_set_option: unknown key or value out of range");
    return TPCG_E_INVALID;
}

// Measurement hooks (see profile.cuh) and the qkdrec_profile_* entry points.
#include <mutex>
#include <vector>

#include "profile.cuh"

namespace qkd {
namespace prof {

static const char *kNames[kNumKinds] = {
    "check_flood_sp_f32", "check_flood_sp_f16", "check_flood_oms_f32", "check_flood_oms_f16",
    "check_flood_oms_i8", "parity_f32", "parity_i8", "var_flood_f32", "var_flood_f16", "var_flood_i8",
    "layer_oms_f32", "layer_oms_f16", "layer_oms_i8", "slice_llr", "quantise", "syndrome",
    "prep", "finish", "woms_check_fwd", "woms_check_bwd", "woms_var", "plan_layered", "layer_qc_tma", "pack", "repack"};

struct Rec {
    int kind;
    cudaEvent_t a, b;
};

static std::mutex g_mu;
static bool g_on = false;
static unsigned long long *g_dev = nullptr;
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_pool;
static thread_local cudaEvent_t t_open[kNumKinds];

static cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

bool on() { return g_on; }

unsigned long long *counters(int kind) { return g_on ? g_dev + 2 * kind : nullptr; }

void start(int kind, cudaStream_t st) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t e = get_event();
    cudaEventRecord(e, st);
    t_open[kind] = e;
}

void stop(int kind, cudaStream_t st) {
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t e = get_event();
    cudaEventRecord(e, st);
    g_recs.push_back(Rec{kind, t_open[kind], e});
}

}  // namespace prof
}  // namespace qkd

using namespace qkd;

extern "C" {

qkdrec_status qkdrec_profile_begin(void) {
    clear_error();
    std::lock_guard<std::mutex> lk(prof::g_mu);
    if (prof::g_on) QKD_FAIL(QKDREC_ERR_ARG, "profiling already on");
    QKD_CUDA(cudaMalloc(&prof::g_dev, sizeof(unsigned long long) * 2 * prof::kNumKinds));
    QKD_CUDA(cudaMemset(prof::g_dev, 0, sizeof(unsigned long long) * 2 * prof::kNumKinds));
    prof::g_recs.clear();
    prof::g_on = true;
    return QKDREC_OK;
}

qkdrec_status qkdrec_profile_end(qkdrec_kernel_stat *stats, int32_t capacity, int32_t *count) {
    clear_error();
    if (!stats || !count || capacity < 0) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(prof::g_mu);
    if (!prof::g_on) QKD_FAIL(QKDREC_ERR_ARG, "profiling is off");
    prof::g_on = false;
    QKD_CUDA(cudaDeviceSynchronize());
    double ms[prof::kNumKinds] = {0};
    int64_t nl[prof::kNumKinds] = {0};
    for (const prof::Rec &r : prof::g_recs) {
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        ms[r.kind] += t;
        nl[r.kind] += 1;
        prof::g_pool.push_back(r.a);
        prof::g_pool.push_back(r.b);
    }
    prof::g_recs.clear();
    unsigned long long h[2 * prof::kNumKinds];
    cudaError_t e = cudaMemcpy(h, prof::g_dev, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(prof::g_dev);
    prof::g_dev = nullptr;
    if (e != cudaSuccess) QKD_FAIL(QKDREC_ERR_CUDA, "counter copy: %s", cudaGetErrorString(e));
    int32_t k = 0;
    for (int i = 0; i < prof::kNumKinds && k < capacity; ++i) {
        if (!nl[i]) continue;
        qkdrec_kernel_stat &s = stats[k++];
        snprintf(s.name, sizeof(s.name), "%s", prof::kNames[i]);
        s.launches = nl[i];
        s.ms = ms[i];
        s.units = (double)h[2 * i];
        s.bytes = (double)h[2 * i + 1];
    }
    *count = k;
    return QKDREC_OK;
}

}  // extern "C"

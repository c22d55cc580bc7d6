// Internal helpers of libqkdrec: status handling, code object, small device utilities.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "qkdrec.h"

namespace qkd {

// Per-thread message of the last failing call.
void set_error(const char *fmt, ...);
void clear_error();

// Return `st` after recording a formatted message.
#define QKD_FAIL(st, ...)                  \
    do {                                   \
        ::qkd::set_error(__VA_ARGS__);     \
        return (st);                       \
    } while (0)

#define QKD_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t err__ = (call);                                                        \
        if (err__ != cudaSuccess)                                                          \
            QKD_FAIL(QKDREC_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(err__),  \
                     __FILE__, __LINE__);                                                  \
    } while (0)

#define QKD_LAUNCHED(name)                                                                 \
    do {                                                                                   \
        cudaError_t err__ = cudaGetLastError();                                            \
        if (err__ != cudaSuccess)                                                          \
            QKD_FAIL(QKDREC_ERR_CUDA, "launch of %s failed: %s", name,                     \
                     cudaGetErrorString(err__));                                           \
    } while (0)

// LLR clip of the channel soft information (nats); paper silent, fixed reading.
constexpr float kLlrClip = 30.0f;
// Sum-product saturation: |q| and the phi-sum are clamped to [kAMin, kAMax].
constexpr float kAMin = 1e-30f;
constexpr float kAMax = 30.0f;
// 6-bit integer min-sum.
constexpr int kQMax = 31;
constexpr int kPMax = 32767;

// The MUFU approximations (PTX ex2/lg2/rcp .approx.ftz): about 2 ulp relative.
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Parity-check matrix with device copies (one per slice; shared by all frames).
struct CodeDev {
    int32_t n = 0, M = 0;
    int64_t E = 0;
    int32_t dc_max = 0, dc_min = 0, dv_max = 0;
    int32_t n_layers = 0;
    uint64_t seed = 0;
    int device = 0;
    // host copies
    std::string note;
    int32_t *h_layer_of = nullptr;  // [M]
    std::vector<int32_t> h_layer_ptr;  // [n_layers+1]
    // device arrays
    int32_t *rp = nullptr;         // [M+1] check -> first edge
    int32_t *ci = nullptr;         // [E]   edge -> variable
    int32_t *vptr = nullptr;       // [n+1] variable -> first slot in vedge
    int32_t *vedge = nullptr;      // [E]   edges of each variable, ascending edge index
    int32_t *layer_ptr = nullptr;  // [n_layers+1]
    int32_t *layer_chk = nullptr;  // [M] checks of each layer, ascending index
    // quasi-cyclic structure (qkdrec_code_set_qc), qc_Z = 0 when absent
    int32_t qc_Z = 0, qc_mb = 0, qc_nb = 0, qc_tma = 0;
    int32_t *qc_shift = nullptr;   // [mb][nb] circulant shifts
};

}  // namespace qkd

struct qkdrec_code_s {
    qkd::CodeDev d;
};

namespace qkd {

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline size_t align_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Number of SMs of the current device (cached per device).
int sm_count();

// Bob's syndromes as the decoder takes them: bytes [F][M], or packed words
// [M][W] (bit f % 32 of word f / 32 of check c at packed[c W + f / 32]).
struct SyndIn {
    const uint8_t *bytes = nullptr;
    const uint32_t *packed = nullptr;
    int64_t W = 0;
};

// qkdrec_decode_batch with either syndrome form (argument checks included).
qkdrec_status decode_batch_impl(qkdrec_code_t code, const float *llr, const SyndIn &synd, int32_t F,
                                const qkdrec_decode_opts *opts, uint8_t *bits_out, int32_t *iters_out,
                                uint8_t *conv_out, float *post_out, void *workspace, size_t workspace_bytes,
                                void *stream);

}  // namespace qkd

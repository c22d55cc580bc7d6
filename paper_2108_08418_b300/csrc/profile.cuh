// Measurement hooks: CUDA events around library launches and device counters
// of algorithmic work, enabled only between qkdrec_profile_begin/end.
#pragma once
#include "common.cuh"

namespace qkd {
namespace prof {

enum Kind {
    kCheckSpF32 = 0, kCheckSpF16, kCheckOmsF32, kCheckOmsF16, kCheckOmsI8,
    kParityF32, kParityI8,
    kVarF32, kVarF16, kVarI8,
    kLayerF32, kLayerF16, kLayerI8,
    kSliceLlr, kQuantise, kSyndrome,
    kPrep, kFinish,
    kWomsFwd, kWomsBwd, kWomsVar, kPlan, kLayerQc, kPack, kRepack,
    kNumKinds
};

// Device counters of kind k: [2k] = units, [2k+1] = bytes.  NULL when off.
unsigned long long *counters(int kind);
bool on();
// Record the start/stop events of one launch of `kind` on `stream` (no-ops when off).
void start(int kind, cudaStream_t stream);
void stop(int kind, cudaStream_t stream);

// RAII bracket around one launch.
struct Scope {
    int kind;
    cudaStream_t st;
    Scope(int k, cudaStream_t s) : kind(k), st(s) { start(k, s); }
    ~Scope() { stop(kind, st); }
};

}  // namespace prof

// Warp-aggregated add of (units, bytes) into a counter pair (p may be NULL).
__device__ __forceinline__ void prof_add(unsigned long long *p, unsigned long long units,
                                         unsigned long long bytes) {
    if (!p) return;
    const unsigned mask = __activemask();
    for (int o = 16; o > 0; o >>= 1) {
        units += __shfl_xor_sync(mask, units, o);
        bytes += __shfl_xor_sync(mask, bytes, o);
    }
    if ((threadIdx.x & 31) == (__ffs(mask) - 1) && units) {
        atomicAdd(p, units);
        atomicAdd(p + 1, bytes);
    }
}

}  // namespace qkd

// Syndrome-based BP decoding of many sub-blocks sharing one parity-check matrix
// (Sec. III-A: N_d decoders loaded with the same matrix; Sec. III-C: BP decoder).
//
// Data layout (frame-interleaved): every per-variable or per-edge quantity is
// stored as [item][Fp] with the frame index fastest, Fp = F rounded up to a
// multiple of 4.  A lane owns V consecutive frames (V = 1 or 4), so the warp
// touches one contiguous run of 32 V elements per edge and the column index of
// an edge is loaded once for all of them.
//
//   llr_i [n][Fp]   channel LLR (float; int8 on the 6-bit grid in integer mode)
//   L     [n][Fp]   posterior (float; int16 in integer mode)
//   msg   [E][Fp]   check-to-variable messages in CSR edge order (float/half/int8)
//   sbits [M][W]    syndrome bits, bit f%32 of word f/32 (W = Fp/32 rounded up)
//   active[Fp]      1 while the frame is decoding
//   unsat [2][W]    bit f%32 of word f/32 set if frame f failed a check in the
//                   stopping test (double-buffered by iteration parity)
//
// One iteration = check kernel + variable kernel.  The check kernel of
// iteration t reads L^(t-1) for every edge anyway, so it also forms the parity
// of the hard decision of L^(t-1) on every check: that is the stopping test of
// the previous iteration, at no extra traffic.  The variable kernel of
// iteration t then retires frames whose test passed (iters = t-1, posterior
// frozen) and updates the others.
//
// Check kernels keep the per-edge state of pass 1 (phi values, or the v->c
// signs) in registers for checks of degree <= DCMAX, so pass 2 only computes
// and stores the outgoing messages; larger degrees use a variant that reloads.
#include <cooperative_groups.h>
#include <cuda.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "profile.cuh"
#include "qkdrec_selftest.h"

namespace qkd {

enum Prec { kF32 = 0, kF16 = 1, kI8 = 2 };
enum Algo { kSP = 0, kOMS = 1 };

constexpr int kCheckWarps = 8;   // warps per check-kernel block
constexpr int kChecksPerWarp = 4;
// edge loads issued together in the first pass of a check (per lane: V frames each)
template <int V> __host__ __device__ constexpr int chunk_of() { return V == 1 ? 8 : 4; }
// frame block of the layout a kernel with V frames per lane runs on: 32 lanes' worth
template <int V> __host__ __device__ constexpr int lgfb_of() { return V == 1 ? 5 : 7; }
constexpr int32_t kMaxFrames = 65535 * 32;  // syndrome packing uses one grid row per 32 frames

// ---------------------------------------------------------------- vector I/O
template <int V> struct VF { float v[V]; };
template <int V> struct VI { int v[V]; };

template <int V> __device__ __forceinline__ VF<V> ldf(const float *p);
template <> __device__ __forceinline__ VF<1> ldf<1>(const float *p) { return VF<1>{{__ldg(p)}}; }
template <> __device__ __forceinline__ VF<4> ldf<4>(const float *p) {
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    return VF<4>{{t.x, t.y, t.z, t.w}};
}
template <int V> __device__ __forceinline__ VF<V> ldf_plain(const float *p);  // coherent (written in-kernel)
template <> __device__ __forceinline__ VF<1> ldf_plain<1>(const float *p) { return VF<1>{{*p}}; }
template <> __device__ __forceinline__ VF<4> ldf_plain<4>(const float *p) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    return VF<4>{{t.x, t.y, t.z, t.w}};
}
template <int V> __device__ __forceinline__ void stf(float *p, const VF<V> &a);
template <> __device__ __forceinline__ void stf<1>(float *p, const VF<1> &a) { *p = a.v[0]; }
template <> __device__ __forceinline__ void stf<4>(float *p, const VF<4> &a) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}

// messages: float or half storage, float arithmetic.  Messages are touched
// once per kernel and the whole array exceeds L2, so they are loaded and
// stored with the streaming (evict-first) hint to keep L2 for the posteriors.
template <int V> __device__ __forceinline__ VF<V> ldm(const float *p);
template <> __device__ __forceinline__ VF<1> ldm<1>(const float *p) { return VF<1>{{__ldcs(p)}}; }
template <> __device__ __forceinline__ VF<4> ldm<4>(const float *p) {
    const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
    return VF<4>{{t.x, t.y, t.z, t.w}};
}
template <int V> __device__ __forceinline__ void stm(float *p, const VF<V> &a);
template <> __device__ __forceinline__ void stm<1>(float *p, const VF<1> &a) { __stcs(p, a.v[0]); }
template <> __device__ __forceinline__ void stm<4>(float *p, const VF<4> &a) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
}
template <int V> __device__ __forceinline__ VF<V> ldm(const __half *p);
template <> __device__ __forceinline__ VF<1> ldm<1>(const __half *p) {
    const unsigned short r = __ldcs(reinterpret_cast<const unsigned short *>(p));
    return VF<1>{{__half2float(__ushort_as_half(r))}};
}
template <> __device__ __forceinline__ VF<4> ldm<4>(const __half *p) {
    uint2 t = __ldcs(reinterpret_cast<const uint2 *>(p));
    const float2 a = __half22float2(*reinterpret_cast<__half2 *>(&t.x));
    const float2 b = __half22float2(*reinterpret_cast<__half2 *>(&t.y));
    return VF<4>{{a.x, a.y, b.x, b.y}};
}
template <int V> __device__ __forceinline__ void stm(__half *p, const VF<V> &a);
template <> __device__ __forceinline__ void stm<1>(__half *p, const VF<1> &a) {
    __stcs(reinterpret_cast<unsigned short *>(p), __half_as_ushort(__float2half_rn(a.v[0])));
}
template <> __device__ __forceinline__ void stm<4>(__half *p, const VF<4> &a) {
    __half2 x = __floats2half2_rn(a.v[0], a.v[1]), y = __floats2half2_rn(a.v[2], a.v[3]);
    uint2 t;
    t.x = *reinterpret_cast<uint32_t *>(&x);
    t.y = *reinterpret_cast<uint32_t *>(&y);
    __stcs(reinterpret_cast<uint2 *>(p), t);
}
// value a message has once stored (FP16 rounding; identity for FP32)
__device__ __forceinline__ float as_stored(float x, const float *) { return x; }
__device__ __forceinline__ float as_stored(float x, const __half *) { return __half2float(__float2half_rn(x)); }

// integer posteriors (int16) and messages / channel values (int8)
template <int V> __device__ __forceinline__ VI<V> ldi16(const int16_t *p);
template <> __device__ __forceinline__ VI<1> ldi16<1>(const int16_t *p) { return VI<1>{{*p}}; }
template <> __device__ __forceinline__ VI<4> ldi16<4>(const int16_t *p) {
    const short4 t = *reinterpret_cast<const short4 *>(p);
    return VI<4>{{t.x, t.y, t.z, t.w}};
}
template <int V> __device__ __forceinline__ void sti16(int16_t *p, const VI<V> &a);
template <> __device__ __forceinline__ void sti16<1>(int16_t *p, const VI<1> &a) { *p = (int16_t)a.v[0]; }
template <> __device__ __forceinline__ void sti16<4>(int16_t *p, const VI<4> &a) {
    *reinterpret_cast<short4 *>(p) = make_short4((short)a.v[0], (short)a.v[1], (short)a.v[2], (short)a.v[3]);
}
template <int V> __device__ __forceinline__ VI<V> ldi8(const int8_t *p);
template <> __device__ __forceinline__ VI<1> ldi8<1>(const int8_t *p) { return VI<1>{{*p}}; }
template <> __device__ __forceinline__ VI<4> ldi8<4>(const int8_t *p) {
    const char4 t = *reinterpret_cast<const char4 *>(p);
    return VI<4>{{t.x, t.y, t.z, t.w}};
}
template <int V> __device__ __forceinline__ VI<V> ldi8s(const int8_t *p);   // streaming (messages)
template <> __device__ __forceinline__ VI<1> ldi8s<1>(const int8_t *p) {
    return VI<1>{{(int)(signed char)__ldcs(reinterpret_cast<const char *>(p))}};
}
template <> __device__ __forceinline__ VI<4> ldi8s<4>(const int8_t *p) {
    const char4 t = __ldcs(reinterpret_cast<const char4 *>(p));
    return VI<4>{{t.x, t.y, t.z, t.w}};
}
template <int V> __device__ __forceinline__ void sti8(int8_t *p, const VI<V> &a);
template <> __device__ __forceinline__ void sti8<1>(int8_t *p, const VI<1> &a) {
    __stcs(reinterpret_cast<char *>(p), (char)a.v[0]);
}
template <> __device__ __forceinline__ void sti8<4>(int8_t *p, const VI<4> &a) {
    __stcs(reinterpret_cast<char4 *>(p), make_char4((signed char)a.v[0], (signed char)a.v[1], (signed char)a.v[2],
                                                    (signed char)a.v[3]));
}

// column index read again in a second pass (volatile: not kept live from pass 1)
__device__ __forceinline__ int32_t ld_index_again(const int32_t *p) {
    int32_t r;
    asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

// active flags of V frames as a bit mask (bit i = frame f0 + i)
template <int V> __device__ __forceinline__ uint32_t active_bits(const uint8_t *p);
template <> __device__ __forceinline__ uint32_t active_bits<1>(const uint8_t *p) { return *p ? 1u : 0u; }
template <> __device__ __forceinline__ uint32_t active_bits<4>(const uint8_t *p) {
    const uint32_t w = *reinterpret_cast<const uint32_t *>(p);
    return (w & 1u) | ((w >> 7) & 2u) | ((w >> 14) & 4u) | ((w >> 21) & 8u);
}

// ------------------------------------------------------------------- phi
// phi(x) = -ln tanh(x/2) = ln coth(x/2) = ln((1 + u)/(1 - u)), u = e^-x, on
// [kAMin, kAMax]; it is its own inverse.  Written from these identities and
// series, evaluated with the MUFU ex2/rcp/lg2 approximations (about 2e-6
// relative), one lg2 shared by the two lower ranges:
//   x >= 2          : u <= 0.135, phi = 2 atanh(u) = 2u (1 + u^2/3 + u^4/5 + u^6/7) + O(u^9);
//   0.03 <= x < 2   : phi = log2((1 + u)/(1 - u)) ln 2, 1 - u >= 0.0296;
//   x < 0.03        : coth(y) y = 1 + y^2/3 - y^4/45 + ..., so with y = x/2
//                     phi = ln(2/x) + x^2/12 - 7 x^4/1440 + O(x^6).
__device__ __forceinline__ float phi_fast(float x) {
    const float kLog2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;
    const float u = ex2_approx(-x * kLog2e);
    const float u2 = u * u;
    const float big = 2.0f * u * (1.0f + u2 * (1.0f / 3.0f + u2 * (0.2f + u2 * (1.0f / 7.0f))));
    const bool small = x < 0.03f;
    const float arg = small ? 0.5f * x : (1.0f + u) * rcp_approx(1.0f - u);
    const float lg = lg2_approx(arg) * kLn2;
    const float x2 = x * x;
    const float low = small ? x2 * (1.0f / 12.0f - x2 * (7.0f / 1440.0f)) - lg : lg;
    return x >= 2.0f ? big : low;
}
__device__ __forceinline__ float phi_clamped(float x) { return phi_fast(fminf(fmaxf(x, kAMin), kAMax)); }

// ------------------------------------------------------------- kernel args
struct DecArgs {
    const int32_t *rp, *ci, *vptr, *vedge;
    const uint32_t *sbits;
    uint8_t *active;
    uint32_t *unsat_cur;    // written by the check kernel of this iteration
    uint32_t *unsat_next;   // cleared by the variable kernel of this iteration
    int32_t *iters_i;
    void *L;
    void *msg;
    const void *llr_i;
    int64_t Fp, FV, W;      // FV = Fp / 4 (the variable kernel's frame vectors)
    int32_t n, M;
    int32_t fvw;            // lanes per check row in check kernels (power of two <= 32)
    int32_t t;              // iteration index (1-based)
    int32_t early_stop;
    int32_t do_msgs;        // 0: parity test only
    float beta;             // OMS offset (float modes)
    unsigned long long *prof;  // (units, bytes) counters of this launch's kernel class, or NULL
    int64_t E;              // edges
    int32_t lgfb;           // log2 of the frame block FB
    const int32_t *blk;     // frame blocks holding at least one decoding frame, ascending
    const int32_t *blk_n;   // their number
    int32_t dstash;         // edges per lane in the shared-memory stash (the code's largest check degree)
};

// Position of (item, frame f) in a frame-block-major array [Fp/FB][items][FB]:
// the FB frames of one item are contiguous and one frame block of all items is
// one contiguous region, so a kernel sweeping the checks of one frame range
// streams through consecutive memory.
__device__ __forceinline__ int64_t fpos(int64_t item, int64_t items, int64_t f, int lgfb) {
    return (((f >> lgfb) * items + item) << lgfb) + (f & ((1 << lgfb) - 1));
}

// Merge the lanes' stopping-test bits (V bits at frame f0) into the 32-frame
// words of this block's frame range, then publish each non-zero word with one
// global atomic.
template <int V>
__device__ __forceinline__ void publish_unsat(uint32_t bits, int64_t f0, int64_t fbase, bool ok,
                                              uint32_t *unsat) {
    __shared__ uint32_t blk[8];
    if (threadIdx.x < 8) blk[threadIdx.x] = 0;
    __syncthreads();
    const int wi = (int)((f0 >> 5) - (fbase >> 5));
    if (ok && bits) atomicOr(&blk[wi], bits << (f0 & 31));
    __syncthreads();
    if (threadIdx.x < 8 && blk[threadIdx.x]) atomicOr(&unsat[(fbase >> 5) + threadIdx.x], blk[threadIdx.x]);
}

// --------------------------------------------------------- float check kernel
// Lane layout: lane = slot * fvw + lfv; the warp serves 32/fvw checks at a time
// (one per slot) over fvw frame vectors of V frames.  blockIdx.x walks check
// groups (so the resident blocks share one range of frames and their
// posterior gathers hit L2), blockIdx.y walks frame ranges.
//
// CACHED (check degree <= kStash): pass 1 keeps what pass 2 needs -- the signs
// of the v->c messages in a bit mask and, for sum-product, phi(|q|) of every
// edge in shared memory ([warp][edge][lane], conflict-free) -- so pass 2 only
// computes and stores the outgoing messages.  Otherwise pass 2 reads the
// posteriors and old messages again.
constexpr int kStash = 32;
// check_flood_sp2: edges per load chunk, and the next chunk's loads issued
// before the current chunk is processed.  Measured on the n = 2^16, 512-frame
// case (B300, 5 iterations): 0.339 ms per launch with chunks of 2 and no
// prefetch at 5 blocks per SM; 0.259 ms with chunks of 4 and prefetch at 4
// blocks per SM (64 registers); chunks of 3 the same, 6 or 8 at 3 blocks slower.
// The first chunk of a warp's next check is fetched during the last chunk of
// the current one: check time +4.5 % throughput at check degree 4, +1.5 % at
// degree 19 (same case), 703.6 -> 682.6 ms per sweep step.
constexpr int kSp2Chunk = 4;
// The same for the flooding min-sum check kernels.  Measured on the same case
// (n = 2^16, 512 frames, 5 iterations): 6-bit integers on 16-bit lanes 0.130 ->
// 0.104 ms per launch with the prefetch; float and FP16 messages (four frames
// per lane) slower with it (0.204 -> 0.315 ms, 0.200 -> 0.248 ms), so off there.
constexpr bool kFloatPrefetch = false;
constexpr bool kI16Prefetch = true;

template <int ALGO, typename MsgT, int V, bool CACHED>
__global__ void __launch_bounds__(kCheckWarps * 32, (ALGO == kSP && V == 1) ? 8 : (ALGO == kOMS && V == 4 ? 4 : 3))
check_flood_f(DecArgs a) {
    extern __shared__ float stash[];  // SP cached: [kCheckWarps][dstash][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw;
    const int slot = lane / fvw, lfv = lane - slot * fvw;
    const float *L = reinterpret_cast<const float *>(a.L);
    MsgT *msg = reinterpret_cast<MsgT *>(a.msg);
    const int64_t nvec = a.Fp / V;
    const uint32_t vmask = (1u << V) - 1u;
    // sum-product, one frame per lane: two loads in flight per lane and the whole
    // SM's 64 warps resident hide the gathers better than deeper chunks at lower
    // occupancy (the kernel is issue-bound, not register-bound)
    constexpr int CH = (ALGO == kSP && V == 1) ? 2 : chunk_of<V>();
    constexpr int LG = lgfb_of<V>();
    constexpr bool SP_STASH = ALGO == kSP && CACHED && V == 1;
    constexpr bool PF = kFloatPrefetch && ALGO == kOMS;   // min-sum forms: next chunk's loads in flight
    float *my = stash + (warp * a.dstash) * 32 + lane;
    unsigned long long units = 0;
    const int32_t nblk = *a.blk_n;
    for (int32_t bi = blockIdx.y; bi < nblk; bi += gridDim.y) {
        const int64_t fb = __ldg(a.blk + bi);
        const int64_t fv = fb * fvw + lfv, f0 = fv * V;
        const bool fv_ok = fv < nvec;
        const int64_t bL = fpos(0, a.n, f0, LG), bM = fpos(0, a.E, f0, LG);  // item 0 of this lane
        const uint32_t act = fv_ok ? active_bits<V>(a.active + f0) : 0u;
        uint32_t unsat_bits = 0;
        if (act) {
            const int nact = __popc(act);
            const int64_t c0 = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
            for (int it = 0; it < kChecksPerWarp; ++it) {
                const int64_t c = c0 + it * slots + slot;
                if (c >= a.M) break;
                const int32_t beg = __ldg(a.rp + c), end = __ldg(a.rp + c + 1), d = end - beg;
                const uint32_t s = (__ldg(a.sbits + c * a.W + (f0 >> 5)) >> (f0 & 31)) & vmask;
                uint32_t par = s;           // syndrome xor hard decisions of L
                uint32_t sg[V];             // bit k: q of edge k negative
                float acc0[V], acc1[V];     // SP: sum of phi except the largest, largest phi
                int32_t arg[V];             // OMS: min1, min2
                for (int i = 0; i < V; ++i) {
                    sg[i] = 0;
                    acc0[i] = ALGO == kSP ? 0.0f : INFINITY;
                    acc1[i] = ALGO == kSP ? 0.0f : INFINITY;
                    arg[i] = -1;
                }
                units += (unsigned long long)d * nact;
                // loads of CH edges are issued together (indices past the last
                // edge are clamped to it), so a warp keeps CH requests in flight
                VF<V> Lw[CH], mw[CH];
                auto fetch = [&](int k0) {
#pragma unroll
                    for (int j = 0; j < CH; ++j) {
                        const int kk = min(k0 + j, d - 1);
                        const int32_t e = beg + kk;
                        const int32_t col = __ldg(a.ci + e);
                        Lw[j] = ldf<V>(L + bL + ((uint32_t)col << LG));
                        if (a.do_msgs) mw[j] = ldm<V>(msg + bM + ((uint32_t)(e) << LG));
                        else for (int i = 0; i < V; ++i) mw[j].v[i] = 0.0f;
                    }
                };
                if (PF) fetch(0);
                for (int k0 = 0; k0 < d; k0 += CH) {
                    VF<V> Lv[CH], mo[CH];
                    if (!PF) fetch(k0);
#pragma unroll
                    for (int j = 0; j < CH; ++j) { Lv[j] = Lw[j]; mo[j] = mw[j]; }
                    // the next chunk's loads go out before this chunk is processed
                    if (PF && k0 + CH < d) fetch(k0 + CH);
#pragma unroll
                    for (int j = 0; j < CH; ++j) {
                        const int k = k0 + j;
                        if (k >= d) break;
                        for (int i = 0; i < V; ++i) {
                            par ^= (uint32_t)(Lv[j].v[i] < 0.0f) << i;   // -0.0 counts as 0
                            const float q = Lv[j].v[i] - mo[j].v[i];
                            if (CACHED && !SP_STASH) sg[i] |= (uint32_t)(q < 0.0f) << k;
                            if (ALGO == kSP) {
                                const float f = phi_clamped(fabsf(q));
                                if (SP_STASH) {
                                    my[k * 32] = q < 0.0f ? -f : f;   // sign of q travels with phi
                                    sg[i] ^= (uint32_t)(q < 0.0f);   // parity of the signs
                                }
                                if (f > acc1[i]) { acc0[i] += acc1[i]; acc1[i] = f; arg[i] = k; }
                                else acc0[i] += f;
                            } else {
                                const float m = fabsf(q);
                                if (m < acc0[i]) { acc1[i] = acc0[i]; acc0[i] = m; arg[i] = k; }
                                else if (m < acc1[i]) acc1[i] = m;
                            }
                        }
                    }
                }
                unsat_bits |= par & act;
                if (!a.do_msgs) continue;
                auto emit = [&](int k, float f_k, bool sneg_k, int i) {
                    float mag;
                    if (ALGO == kSP) {
                        const float ex = (k == arg[i]) ? acc0[i] : acc0[i] + (acc1[i] - f_k);
                        mag = phi_clamped(ex);
                    } else {
                        mag = fmaxf(((k == arg[i]) ? acc1[i] : acc0[i]) - a.beta, 0.0f);
                    }
                    return sneg_k ? -mag : mag;
                };
                if (SP_STASH) {
                    const uint32_t neg = (s ^ sg[0]) & 1u;   // syndrome xor all signs of q
                    for (int k = 0; k < d; ++k) {
                        const float fs = my[k * 32];
                        VF<V> mn;
                        mn.v[0] = emit(k, fabsf(fs), neg ^ (__float_as_uint(fs) >> 31), 0);
                        stm<V>(msg + bM + ((uint32_t)(beg + k) << LG), mn);
                    }
                } else if (CACHED && ALGO != kSP) {
                    uint32_t neg = s;       // syndrome xor all signs of q
                    for (int i = 0; i < V; ++i) neg ^= (uint32_t)(__popc(sg[i]) & 1) << i;
                    for (int k = 0; k < d; ++k) {
                        VF<V> mn;
                        for (int i = 0; i < V; ++i)
                            mn.v[i] = emit(k, 0.0f, ((neg >> i) & 1u) ^ ((sg[i] >> k) & 1u), i);
                        stm<V>(msg + bM + ((uint32_t)(beg + k) << LG), mn);
                    }
                } else {
                    // signs and phi values again from memory
                    uint32_t negall = s;
                    for (int k = 0; k < d; ++k) {
                        const int32_t e = beg + k;
                        const VF<V> Lv = ldf<V>(L + bL + ((uint32_t)__ldg(a.ci + e) << LG));
                        const VF<V> mo = ldm<V>(msg + bM + ((uint32_t)(e) << LG));
                        for (int i = 0; i < V; ++i) negall ^= (uint32_t)(Lv.v[i] - mo.v[i] < 0.0f) << i;
                    }
                    for (int k = 0; k < d; ++k) {
                        const int32_t e = beg + k;
                        const VF<V> Lv = ldf<V>(L + bL + ((uint32_t)__ldg(a.ci + e) << LG));
                        MsgT *mp = msg + bM + ((uint32_t)(e) << LG);
                        const VF<V> mo = ldm<V>(mp);
                        VF<V> mn;
                        for (int i = 0; i < V; ++i) {
                            const float q = Lv.v[i] - mo.v[i];
                            const float f = ALGO == kSP ? phi_clamped(fabsf(q)) : 0.0f;
                            mn.v[i] = emit(k, f, ((negall >> i) & 1u) ^ (q < 0.0f), i);
                        }
                        stm<V>(mp, mn);
                    }
                }
            }
        }
        if (a.early_stop || !a.do_msgs)
            publish_unsat<V>(unsat_bits, f0, fb * fvw * V, fv_ok, a.unsat_cur);
    }
    // messages read + written and the posterior gathered, per active edge-frame
    prof_add(a.prof, units, units * (a.do_msgs ? 2 * sizeof(MsgT) + 4 : 4));
}

// ------------------------------ sum-product check kernel, two frames per lane
// phi of two values at once: the polynomial and product steps in packed FP32x2
// arithmetic (one instruction for both), the MUFU approximations per value.
// The same identities as phi_fast, with the small-argument range folded into
// the logarithmic one: below 0.1, 1 - e^-x is formed from its series
// x (1 - x/2 + x^2/6 - x^3/24 + x^4/120) (relative truncation < 1.4e-8), so
//   x >= 2 : phi = 2u (1 + u^2/3 + u^4/5 + u^6/7),  u = e^-x,
//   x <  2 : phi = ln((1 + u) / (1 - u)).
__device__ __forceinline__ float2 phi2(float2 x) {
    const float kLog2e = 1.4426950408889634f, kLn2 = 0.6931471805599453f;
    const float2 t = __fmul2_rn(x, f2(-kLog2e));
    const float2 u = make_float2(ex2_approx(t.x), ex2_approx(t.y));
    const float2 u2 = __fmul2_rn(u, u);
    float2 p = __ffma2_rn(u2, f2(1.0f / 7.0f), f2(0.2f));
    p = __ffma2_rn(u2, p, f2(1.0f / 3.0f));
    p = __ffma2_rn(u2, p, f2(1.0f));
    const float2 big = __fmul2_rn(__fadd2_rn(u, u), p);
    float2 sr = __ffma2_rn(x, f2(1.0f / 120.0f), f2(-1.0f / 24.0f));
    sr = __ffma2_rn(x, sr, f2(1.0f / 6.0f));
    sr = __ffma2_rn(x, sr, f2(-0.5f));
    sr = __ffma2_rn(x, sr, f2(1.0f));
    const float2 dser = __fmul2_rn(x, sr);
    const float2 dsub = __ffma2_rn(u, f2(-1.0f), f2(1.0f));
    const float2 r = make_float2(rcp_approx(x.x < 0.1f ? dser.x : dsub.x), rcp_approx(x.y < 0.1f ? dser.y : dsub.y));
    const float2 ar = __ffma2_rn(u, r, r);                       // (1 + u) / (1 - u)
    const float2 mid = __fmul2_rn(make_float2(lg2_approx(ar.x), lg2_approx(ar.y)), f2(kLn2));
    return make_float2(x.x >= 2.0f ? big.x : mid.x, x.y >= 2.0f ? big.y : mid.y);
}
__device__ __forceinline__ uint32_t fbits(float x) { return __float_as_uint(x); }

// The sum-product check update of check_flood_f<kSP, float, 1, true> on the
// same 32-frame-block layout, with each lane holding two frames of a block:
// half-warp h serves listed block 2 b + h, lane l of it frames 2l, 2l + 1, so a
// warp moves one 8-byte value per lane per edge and shares the edge's column
// index and address arithmetic between two frames.  Per check and frame, pass 1
// keeps sum-except-largest and largest of phi(|q|) in the form
//   acc0 += min(f, acc1),  acc1 = max(f, acc1)
// (no argmax: for the largest edge acc0 + (acc1 - f) = acc0 exactly), and
// stashes phi(|q|) carrying the sign of q in shared memory; the signs, the
// hard decisions' parity and the syndrome are XORs of whole words.  Posteriors
// are made +0.0 for -0.0 first (L + 0), so a sign bit is a hard decision and
// q = L - m (never -0.0 then) carries sgn(0) = +1.
template <int CH>
__global__ void __launch_bounds__(kCheckWarps * 32, 4)
check_flood_sp2(DecArgs a) {
    extern __shared__ float2 stash2[];   // [kCheckWarps][dstash][32]
    __shared__ uint32_t blkw[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = lane >> 4, hl = lane & 15;
    const float *L = reinterpret_cast<const float *>(a.L);
    float *msg = reinterpret_cast<float *>(a.msg);
    constexpr int LG = 5;
    float2 *my = stash2 + (warp * a.dstash) * 32 + lane;
    unsigned long long units = 0;
    const int32_t nblk = *a.blk_n;
    const int64_t c0 = ((int64_t)blockIdx.x * kCheckWarps + warp) * kChecksPerWarp;
    for (int32_t bp = blockIdx.y; 2 * bp < nblk; bp += gridDim.y) {
        const int32_t bi = 2 * bp + half;
        const int64_t fb = bi < nblk ? __ldg(a.blk + bi) : -1;
        const int64_t f0 = (fb << LG) + 2 * hl;
        uint32_t act = 0;
        if (fb >= 0) {
            const uint32_t w = *reinterpret_cast<const uint16_t *>(a.active + f0);
            act = (w & 1u) | ((w >> 7) & 2u);
        }
        uint32_t unsat_bits = 0;
        if (act) {
            const int nact = __popc(act);
            const int64_t bL = fpos(0, a.n, f0, LG), bM = fpos(0, a.E, f0, LG);
            // the next chunk's loads go out before a chunk is processed; after a
            // check's last chunk, the first chunk of this warp's next check (its
            // edges and messages are disjoint from this check's, the posteriors
            // read-only here), so a check of a few edges still overlaps its
            // gather with the previous check's work
            float2 Lv[CH], mo[CH];
            auto fetch = [&](int32_t fbeg, int32_t fd, int k0) {
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int32_t e = fbeg + min(k0 + j, fd - 1);
                    const int32_t col = __ldg(a.ci + e);
                    Lv[j] = __ldg(reinterpret_cast<const float2 *>(L + bL + ((uint32_t)col << LG)));
                    mo[j] = __ldcs(reinterpret_cast<const float2 *>(msg + bM + ((uint32_t)e << LG)));
                }
            };
            int32_t nbeg = 0, nd = 0;
            if (c0 < a.M) {
                nbeg = __ldg(a.rp + c0);
                nd = __ldg(a.rp + c0 + 1) - nbeg;
                if (nd > 0) fetch(nbeg, nd, 0);
            }
            for (int it = 0; it < kChecksPerWarp; ++it) {
                const int64_t c = c0 + it;
                if (c >= a.M) break;
                const int32_t beg = nbeg, d = nd;
                const bool more = it + 1 < kChecksPerWarp && c + 1 < a.M;
                if (more) {
                    nbeg = __ldg(a.rp + c + 1);
                    nd = __ldg(a.rp + c + 2) - nbeg;
                }
                const uint32_t s = (__ldg(a.sbits + c * a.W + (f0 >> 5)) >> (f0 & 31)) & 3u;
                uint32_t px = 0, py = 0, sx = 0, sy = 0;     // xor of L words, of q words
                float2 acc0 = f2(0.0f), acc1 = f2(0.0f);
                units += (unsigned long long)d * nact;
                for (int k0 = 0; k0 < d; k0 += CH) {
                    float2 Lc2[CH], mc2[CH];
#pragma unroll
                    for (int j = 0; j < CH; ++j) { Lc2[j] = Lv[j]; mc2[j] = mo[j]; }
                    if (k0 + CH < d) fetch(beg, d, k0 + CH);
                    else if (more && nd > 0) fetch(nbeg, nd, 0);
#pragma unroll
                    for (int j = 0; j < CH; ++j) {
                        const int k = k0 + j;
                        if (k >= d) break;
                        const float2 Lc = __fadd2_rn(Lc2[j], f2(0.0f));
                        px ^= fbits(Lc.x);
                        py ^= fbits(Lc.y);
                        const float2 q = __ffma2_rn(mc2[j], f2(-1.0f), Lc);
                        sx ^= fbits(q.x);
                        sy ^= fbits(q.y);
                        const float2 aq = make_float2(fmaxf(fminf(fabsf(q.x), kAMax), kAMin),
                                                      fmaxf(fminf(fabsf(q.y), kAMax), kAMin));
                        const float2 f = phi2(aq);
                        my[k * 32] = make_float2(__uint_as_float(fbits(f.x) | (fbits(q.x) & 0x80000000u)),
                                                 __uint_as_float(fbits(f.y) | (fbits(q.y) & 0x80000000u)));
                        acc0 = __fadd2_rn(acc0, make_float2(fminf(f.x, acc1.x), fminf(f.y, acc1.y)));
                        acc1 = make_float2(fmaxf(f.x, acc1.x), fmaxf(f.y, acc1.y));
                    }
                }
                unsat_bits |= (s ^ (px >> 31) ^ ((py >> 30) & 2u)) & act;
                // syndrome xor the signs of all q, in the sign bit of each frame's word
                const uint32_t nx = (s << 31) ^ sx, ny = ((s & 2u) << 30) ^ sy;
                for (int k = 0; k < d; ++k) {
                    const float2 fs = my[k * 32];
                    const float2 f = make_float2(fabsf(fs.x), fabsf(fs.y));
                    const float2 ex = __fadd2_rn(acc0, __ffma2_rn(f, f2(-1.0f), acc1));
                    const float2 mg = phi2(make_float2(fminf(ex.x, kAMax), fminf(ex.y, kAMax)));
                    const float2 mn = make_float2(__uint_as_float(fbits(mg.x) | ((fbits(fs.x) ^ nx) & 0x80000000u)),
                                                  __uint_as_float(fbits(mg.y) | ((fbits(fs.y) ^ ny) & 0x80000000u)));
                    __stcs(reinterpret_cast<float2 *>(msg + bM + ((uint32_t)(beg + k) << LG)), mn);
                }
            }
        }
        if (a.early_stop) {
            // merge the stopping-test bits of each half-warp's block, then one
            // global atomic per block
            uint32_t v = unsat_bits << (2 * hl);
            for (int o = 8; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
            if (threadIdx.x < 2) blkw[threadIdx.x] = 0;
            __syncthreads();
            if (hl == 0 && v) atomicOr(&blkw[half], v);
            __syncthreads();
            if (threadIdx.x < 2 && blkw[threadIdx.x]) {
                const int32_t bj = 2 * bp + (int32_t)threadIdx.x;
                atomicOr(&a.unsat_cur[__ldg(a.blk + bj)], blkw[threadIdx.x]);
            }
            __syncthreads();
        }
    }
    prof_add(a.prof, units, units * 12);
}

// ----------------------------------------------------- integer check kernel
template <int V, int DCMAX>
__global__ void __launch_bounds__(kCheckWarps * 32)
check_flood_i(DecArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw;
    const int slot = lane / fvw, lfv = lane - slot * fvw;
    const int16_t *L = reinterpret_cast<const int16_t *>(a.L);
    int8_t *msg = reinterpret_cast<int8_t *>(a.msg);
    const int64_t nvec = a.Fp / V;
    const uint32_t vmask = (1u << V) - 1u;
    constexpr int CH = V == 4 ? 2 : chunk_of<V>();   // measured: two 4-frame loads in flight per lane
    constexpr int LG = lgfb_of<V>();
    unsigned long long units = 0;
    const int32_t nblk = *a.blk_n;
    for (int32_t bi = blockIdx.y; bi < nblk; bi += gridDim.y) {
        const int64_t fb = __ldg(a.blk + bi);
        const int64_t fv = fb * fvw + lfv, f0 = fv * V;
        const bool fv_ok = fv < nvec;
        const int64_t bL = fpos(0, a.n, f0, LG), bM = fpos(0, a.E, f0, LG);  // item 0 of this lane
        const uint32_t act = fv_ok ? active_bits<V>(a.active + f0) : 0u;
        uint32_t unsat_bits = 0;
        if (act) {
            const int nact = __popc(act);
            const int64_t c0 = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
            for (int it = 0; it < kChecksPerWarp; ++it) {
                const int64_t c = c0 + it * slots + slot;
                if (c >= a.M) break;
                const int32_t beg = __ldg(a.rp + c), end = __ldg(a.rp + c + 1), d = end - beg;
                const uint32_t s = (__ldg(a.sbits + c * a.W + (f0 >> 5)) >> (f0 & 31)) & vmask;
                uint32_t par = s, sg[V];
                int mn1[V], mn2[V], arg[V];
                for (int i = 0; i < V; ++i) { sg[i] = 0; mn1[i] = 1 << 20; mn2[i] = 1 << 20; arg[i] = -1; }
                units += (unsigned long long)d * nact;
                auto visit = [&](int k, const VI<V> &Lv, const VI<V> &mo) {
                    for (int i = 0; i < V; ++i) {
                        par ^= (uint32_t)(Lv.v[i] < 0) << i;
                        const int q = max(min(Lv.v[i] - mo.v[i], kQMax), -kQMax);
                        if (k < 32) sg[i] |= (uint32_t)(q < 0) << k;
                        const int m = q < 0 ? -q : q;
                        if (m < mn1[i]) { mn2[i] = mn1[i]; mn1[i] = m; arg[i] = k; }
                        else if (m < mn2[i]) mn2[i] = m;
                    }
                };
                auto load = [&](int k, VI<V> &Lv, VI<V> &mo) {
                    const int32_t e = beg + k;
                    Lv = ldi16<V>(L + bL + ((uint32_t)(__ldg(a.ci + e)) << LG));
                    if (a.do_msgs) mo = ldi8s<V>(msg + bM + ((uint32_t)(e) << LG));
                    else for (int i = 0; i < V; ++i) mo.v[i] = 0;
                };
                for (int k0 = 0; k0 < d; k0 += CH) {
                    VI<V> Lv[CH], mo[CH];
#pragma unroll
                    for (int j = 0; j < CH; ++j) load(min(k0 + j, d - 1), Lv[j], mo[j]);
#pragma unroll
                    for (int j = 0; j < CH; ++j)
                        if (k0 + j < d) visit(k0 + j, Lv[j], mo[j]);
                }
                unsat_bits |= par & act;
                if (!a.do_msgs) continue;
                auto emit = [&](int k, bool sneg, int i) {
                    const int mag = max(((k == arg[i]) ? mn2[i] : mn1[i]) - 1, 0);
                    return sneg ? -mag : mag;
                };
                if (DCMAX > 0) {
                    // the outgoing message needs only the signs kept in pass 1
                    uint32_t neg = s;
                    for (int i = 0; i < V; ++i) neg ^= (uint32_t)(__popc(sg[i]) & 1) << i;
                    for (int k = 0; k < d; ++k) {
                        VI<V> mn;
                        for (int i = 0; i < V; ++i) mn.v[i] = emit(k, ((neg >> i) & 1u) ^ ((sg[i] >> k) & 1u), i);
                        sti8<V>(msg + bM + ((uint32_t)(beg + k) << LG), mn);
                    }
                } else {
                    uint32_t negall = s;
                    for (int k = 0; k < d; ++k) {
                        VI<V> Lv, mo;
                        load(k, Lv, mo);
                        for (int i = 0; i < V; ++i)
                            negall ^= (uint32_t)(max(min(Lv.v[i] - mo.v[i], kQMax), -kQMax) < 0) << i;
                    }
                    for (int k = 0; k < d; ++k) {
                        VI<V> Lv, mo, mn;
                        load(k, Lv, mo);
                        for (int i = 0; i < V; ++i) {
                            const int q = max(min(Lv.v[i] - mo.v[i], kQMax), -kQMax);
                            mn.v[i] = emit(k, ((negall >> i) & 1u) ^ (q < 0), i);
                        }
                        sti8<V>(msg + bM + ((uint32_t)(beg + k) << LG), mn);
                    }
                }
            }
        }
        if (a.early_stop || !a.do_msgs)
            publish_unsat<V>(unsat_bits, f0, fb * fvw * V, fv_ok, a.unsat_cur);
    }
    prof_add(a.prof, units, units * (a.do_msgs ? 4 : 2));
}

// ------------------------------------------ integer check kernel, 16-bit lanes
// The same offset min-sum check update as check_flood_i<4, 32>, bit for bit,
// with a lane's four frames held as two pairs of 16-bit lanes (s16x2: frames
// 0-1 and 2-3), so that one min/max/add serves two frames.  Identities used
// (|L| <= 31 (dv + 1) and |m| <= 31, so L - m fits a 16-bit lane):
//   t = ~L + m = -q - 1 per lane, so q = ~t, -q = t + 1, sign(q) = NOT sign(t);
//   the second minimum is needed exactly where |q_k| equals the minimum (if
//   another edge shares the minimum, the second minimum equals it), so no
//   argmin is tracked;  max(x - 1, 0) commutes with that choice, so the
//   offset is applied to the two minima once per check.
// Pass 1 keeps |q| with the sign of q in bit 7 of one byte per frame
// (four frames in a word) in shared memory for pass 2.
__device__ __forceinline__ uint32_t vmin_s16(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("min.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t vmax_s16(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("max.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t vmin_u16(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t vadd_16(uint32_t a, uint32_t b) {   // lane-wise, no carry between lanes
    uint32_t r;
    asm("add.s16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(sel));
    return r;
}
// sign bits 15 and 31 of a pair -> frame bits (b0 -> bit `lo`, b1 -> bit lo + 1)
__device__ __forceinline__ uint32_t pair_signs(uint32_t x, int lo) {
    return (((x >> 15) & 1u) | ((x >> 30) & 2u)) << lo;
}

__global__ void __launch_bounds__(kCheckWarps * 32, 4)
check_flood_i16x2(DecArgs a) {
    extern __shared__ uint32_t istash[];   // [kCheckWarps][dstash][32]: per edge, four frames of |q| | sign << 7
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw;
    const int slot = lane / fvw, lfv = lane - slot * fvw;
    const int16_t *L = reinterpret_cast<const int16_t *>(a.L);
    int8_t *msg = reinterpret_cast<int8_t *>(a.msg);
    const int64_t nvec = a.Fp / 4;
    constexpr int CH = 4;
    constexpr int LG = lgfb_of<4>();
    constexpr uint32_t kOnes = 0x00010001u, kMax = 0x001F001Fu;   // 1 and kQMax in both lanes
    uint32_t *my = istash + (warp * a.dstash) * 32 + lane;
    unsigned long long units = 0;
    const int32_t nblk = *a.blk_n;
    for (int32_t bi = blockIdx.y; bi < nblk; bi += gridDim.y) {
        const int64_t fb = __ldg(a.blk + bi);
        const int64_t fv = fb * fvw + lfv, f0 = fv * 4;
        const bool fv_ok = fv < nvec;
        const int64_t bL = fpos(0, a.n, f0, LG), bM = fpos(0, a.E, f0, LG);
        const uint32_t act = fv_ok ? active_bits<4>(a.active + f0) : 0u;
        uint32_t unsat_bits = 0;
        if (act) {
            const int nact = __popc(act);
            const int64_t c0 = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
            for (int it = 0; it < kChecksPerWarp; ++it) {
                const int64_t c = c0 + it * slots + slot;
                if (c >= a.M) break;
                const int32_t beg = __ldg(a.rp + c), end = __ldg(a.rp + c + 1), d = end - beg;
                const uint32_t s = (__ldg(a.sbits + c * a.W + (f0 >> 5)) >> (f0 & 31)) & 0xFu;
                uint32_t pA = 0, pB = 0;                 // xor of L: hard decisions in the sign bits
                uint32_t nA = 0, nB = 0;                 // xor of t = -q - 1
                uint32_t m1A = 0x7FFF7FFFu, m1B = 0x7FFF7FFFu, m2A = 0x7FFF7FFFu, m2B = 0x7FFF7FFFu;
                units += (unsigned long long)d * nact;
                auto edge = [&](uint32_t Lx, uint32_t mx, uint32_t &m1, uint32_t &m2, uint32_t &n) {
                    const uint32_t t = vadd_16(~Lx, mx);
                    const uint32_t q = ~t;
                    const uint32_t aq = vmin_s16(vmax_s16(q, vadd_16(t, kOnes)), kMax);   // |clamp(q)|
                    n ^= t;
                    m2 = vmin_s16(m2, vmax_s16(m1, aq));
                    m1 = vmin_s16(m1, aq);
                    return aq | ((q >> 8) & 0x00800080u);
                };
                uint2 Lw[CH];
                uint32_t mw[CH];
                auto fetch = [&](int k0) {
#pragma unroll
                    for (int j = 0; j < CH; ++j) {
                        const int32_t e = beg + min(k0 + j, d - 1);
                        Lw[j] = *reinterpret_cast<const uint2 *>(L + bL + ((uint32_t)__ldg(a.ci + e) << LG));
                        mw[j] = a.do_msgs ? __ldcs(reinterpret_cast<const unsigned int *>(msg + bM + ((uint32_t)e << LG)))
                                          : 0u;
                    }
                };
                if (kI16Prefetch) fetch(0);
                for (int k0 = 0; k0 < d; k0 += CH) {
                    uint2 Lc[CH];
                    uint32_t mc[CH];
                    if (!kI16Prefetch) fetch(k0);
#pragma unroll
                    for (int j = 0; j < CH; ++j) { Lc[j] = Lw[j]; mc[j] = mw[j]; }
                    // the next chunk's loads go out before this chunk is processed
                    if (kI16Prefetch && k0 + CH < d) fetch(k0 + CH);
#pragma unroll
                    for (int j = 0; j < CH; ++j) {
                        const int k = k0 + j;
                        if (k >= d) break;
                        pA ^= Lc[j].x;
                        pB ^= Lc[j].y;
                        const uint32_t sa = edge(Lc[j].x, prmt(mc[j], 0u, 0x9180u), m1A, m2A, nA);
                        const uint32_t sb = edge(Lc[j].y, prmt(mc[j], 0u, 0xB3A2u), m1B, m2B, nB);
                        my[k * 32] = prmt(sa, sb, 0x6420u);
                    }
                }
                unsat_bits |= (s ^ pair_signs(pA, 0) ^ pair_signs(pB, 2)) & act;
                if (!a.do_msgs) continue;
                // per frame: syndrome xor the signs of all q (sign(q) = NOT sign(t))
                const uint32_t neg = s ^ pair_signs(nA, 0) ^ pair_signs(nB, 2) ^ ((d & 1) ? 0xFu : 0u);
                const uint32_t NA = ((neg & 1u) << 7) | ((neg & 2u) << 22), NB = ((neg & 4u) << 5) | ((neg & 8u) << 20);
                const uint32_t o1A = vmax_s16(vadd_16(m1A, 0xFFFFFFFFu), 0u), o2A = vmax_s16(vadd_16(m2A, 0xFFFFFFFFu), 0u);
                const uint32_t o1B = vmax_s16(vadd_16(m1B, 0xFFFFFFFFu), 0u), o2B = vmax_s16(vadd_16(m2B, 0xFFFFFFFFu), 0u);
                auto out = [&](uint32_t w, uint32_t m1, uint32_t o1, uint32_t o2, uint32_t N) {
                    const uint32_t u = vmin_u16((w & kMax) - m1, kOnes) ^ kOnes;   // 1 where |q| is the minimum
                    const uint32_t mag = vmin_u16(o2, u * 0x7FFFu + o1);          // u ? o2 : o1
                    const uint32_t sg = ((w ^ N) >> 7) & kOnes;                     // 1 where the message is negative
                    return vadd_16(mag ^ (sg * 0xFFFFu), sg);
                };
                for (int k = 0; k < d; ++k) {
                    const uint32_t w = my[k * 32];
                    const uint32_t rA = out(prmt(w, 0u, 0x4140u), m1A, o1A, o2A, NA);
                    const uint32_t rB = out(prmt(w, 0u, 0x4342u), m1B, o1B, o2B, NB);
                    __stcs(reinterpret_cast<unsigned int *>(msg + bM + ((uint32_t)(beg + k) << LG)), prmt(rA, rB, 0x6420u));
                }
            }
        }
        if (a.early_stop || !a.do_msgs)
            publish_unsat<4>(unsat_bits, f0, fb * fvw * 4, fv_ok, a.unsat_cur);
    }
    prof_add(a.prof, units, units * (a.do_msgs ? 4 : 2));
}

// ------------------------------------------------------------ variable kernels
// Retire frames whose stopping test passed on L^(t-1); update the rest:
// L_v = llr_v + sum of the messages on the edges of v (ascending edge order).
// Four frames per lane.
template <int PREC>
__global__ void __launch_bounds__(256) var_flood(DecArgs a) {
    // items: (listed frame block, variable, frame vector of the block), the
    // vectors of one variable and block contiguous in memory
    const int64_t fbv = (int64_t)1 << (a.lgfb - 2);      // frame vectors per block
    const int64_t per_blk = (int64_t)a.n * fbv;
    const int64_t total = per_blk * *a.blk_n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // per updated variable-frame: its messages, its channel LLR, the new posterior
    constexpr unsigned ms = PREC == kF32 ? 4 : (PREC == kF16 ? 2 : 1);
    constexpr unsigned cs = PREC == kI8 ? 1 : 4, ls = PREC == kI8 ? 2 : 4;
    unsigned long long units = 0, bytes = 0;
    for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < total; item += stride) {
        const int64_t bi = item / per_blk, r = item - bi * per_blk;
        const int64_t v = r / fbv, fv = (int64_t)__ldg(a.blk + bi) * fbv + (r - v * fbv), f0 = 4 * fv;
        if (f0 >= a.Fp) continue;
        const int64_t bL = fpos(0, a.n, f0, a.lgfb), bM = fpos(0, a.E, f0, a.lgfb);
        if (v == 0 && (fv & 7) == 0 && a.early_stop) a.unsat_next[fv >> 3] = 0;  // next test starts clear
        const uint32_t act = active_bits<4>(a.active + f0);
        if (!act) continue;
        const uint32_t u = a.early_stop ? (__ldcg(a.unsat_cur + (f0 >> 5)) >> (f0 & 31)) & 0xfu : 0xfu;
        const uint32_t done = a.early_stop ? (act & ~u) : 0u;  // frames retiring now
        const uint32_t upd = act & ~done;                      // frames to update
        if (v == 0)
            for (int i = 0; i < 4; ++i)
                if ((done >> i) & 1u) {
                    a.active[f0 + i] = 0;
                    a.iters_i[f0 + i] = a.t - 1;
                }
        if (!upd) continue;
        const int32_t vb = __ldg(a.vptr + v), ve = __ldg(a.vptr + v + 1);
        const int64_t pv = bL + ((int64_t)(v) << a.lgfb);
        const unsigned nu = __popc(upd);
        units += nu;
        bytes += (unsigned long long)nu * ((ve - vb) * ms + cs + ls);
        if (PREC != kI8) {
            float *L = reinterpret_cast<float *>(a.L);
            VF<4> s = ldf<4>(reinterpret_cast<const float *>(a.llr_i) + pv);
            for (int32_t k = vb; k < ve; ++k) {
                const int64_t e = __ldg(a.vedge + k);
                VF<4> m;
                if (PREC == kF32) m = ldm<4>(reinterpret_cast<const float *>(a.msg) + bM + ((int64_t)(e) << a.lgfb));
                else m = ldm<4>(reinterpret_cast<const __half *>(a.msg) + bM + ((int64_t)(e) << a.lgfb));
                for (int i = 0; i < 4; ++i) s.v[i] += m.v[i];
            }
            if (upd != 0xfu) {
                const VF<4> old = ldf_plain<4>(L + pv);
                for (int i = 0; i < 4; ++i)
                    if (!((upd >> i) & 1u)) s.v[i] = old.v[i];
            }
            stf<4>(L + pv, s);
        } else {
            int16_t *L = reinterpret_cast<int16_t *>(a.L);
            VI<4> s = ldi8<4>(reinterpret_cast<const int8_t *>(a.llr_i) + pv);
            for (int32_t k = vb; k < ve; ++k) {
                const int64_t e = __ldg(a.vedge + k);
                const VI<4> m = ldi8s<4>(reinterpret_cast<const int8_t *>(a.msg) + bM + ((int64_t)(e) << a.lgfb));
                for (int i = 0; i < 4; ++i) s.v[i] = max(min(s.v[i] + m.v[i], kPMax), -kPMax);
            }
            if (upd != 0xfu) {
                const VI<4> old = ldi16<4>(L + pv);
                for (int i = 0; i < 4; ++i)
                    if (!((upd >> i) & 1u)) s.v[i] = old.v[i];
            }
            sti16<4>(L + pv, s);
        }
    }
    prof_add(a.prof, units, bytes);
}

// Integer flooding, variable side, 16 frames per thread as eight pairs of
// 16-bit lanes: thread (listed frame block on y, (variable, group of 16 frames)
// on x).  Sums are the same as var_flood<kI8>'s: with |L| <= kQMax (dv + 1)
// the saturation at kPMax is never reached, so plain lane-wise adds agree.
__global__ void __launch_bounds__(256) var_flood_i8x16(DecArgs a) {
    constexpr int LG = lgfb_of<4>();                   // 128-frame blocks: 8 groups of 16
    const int64_t items = (int64_t)a.n * 8;
    const int16_t *Lc = reinterpret_cast<const int16_t *>(a.L);
    int16_t *L = reinterpret_cast<int16_t *>(a.L);
    const int8_t *llr = reinterpret_cast<const int8_t *>(a.llr_i);
    const int8_t *msg = reinterpret_cast<const int8_t *>(a.msg);
    unsigned long long units = 0, bytes = 0;
    const int32_t nblk = *a.blk_n;
    for (int32_t bi = blockIdx.y; bi < nblk; bi += gridDim.y) {
        const int64_t fb = __ldg(a.blk + bi);
        for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < items;
             idx += (int64_t)gridDim.x * blockDim.x) {
            const int64_t v = idx >> 3, f0 = (fb << LG) + ((idx & 7) << 4);
            const int64_t bL = fpos(0, a.n, f0, LG), bM = fpos(0, a.E, f0, LG);
            if (v == 0 && (f0 & 31) == 0 && a.early_stop) a.unsat_next[f0 >> 5] = 0;   // next test starts clear
            const uint4 aw = *reinterpret_cast<const uint4 *>(a.active + f0);
            const uint32_t act = active_bits<4>(reinterpret_cast<const uint8_t *>(&aw.x)) |
                                 (active_bits<4>(reinterpret_cast<const uint8_t *>(&aw.y)) << 4) |
                                 (active_bits<4>(reinterpret_cast<const uint8_t *>(&aw.z)) << 8) |
                                 (active_bits<4>(reinterpret_cast<const uint8_t *>(&aw.w)) << 12);
            if (!act) continue;
            const uint32_t u = a.early_stop ? (__ldcg(a.unsat_cur + (f0 >> 5)) >> (f0 & 31)) & 0xffffu : 0xffffu;
            const uint32_t done = a.early_stop ? (act & ~u) : 0u;
            const uint32_t upd = act & ~done;
            if (v == 0)
                for (uint32_t r = done; r; r &= r - 1) {
                    const int i = __ffs(r) - 1;
                    a.active[f0 + i] = 0;
                    a.iters_i[f0 + i] = a.t - 1;
                }
            if (!upd) continue;
            const int32_t vb = __ldg(a.vptr + v), ve = __ldg(a.vptr + v + 1);
            const int64_t pv = bL + (v << LG);
            const unsigned nu = __popc(upd);
            units += nu;
            bytes += (unsigned long long)nu * ((ve - vb) + 1 + 2);
            uint32_t acc[8];
            {
                const uint4 c = __ldg(reinterpret_cast<const uint4 *>(llr + pv));
                const uint32_t cw[4] = {c.x, c.y, c.z, c.w};
                for (int w = 0; w < 4; ++w) {
                    acc[2 * w] = prmt(cw[w], 0u, 0x9180u);       // frames 4w, 4w+1 sign-extended
                    acc[2 * w + 1] = prmt(cw[w], 0u, 0xB3A2u);   // frames 4w+2, 4w+3
                }
            }
            // edges in chunks of four: the index loads, then the message loads,
            // are issued together (a variable of degree 3 is one chunk)
            for (int32_t k0 = vb; k0 < ve; k0 += 4) {
                int32_t e[4];
                uint4 m[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) e[j] = __ldg(a.vedge + min(k0 + j, ve - 1));
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (k0 + j < ve) m[j] = __ldcs(reinterpret_cast<const uint4 *>(msg + bM + ((int64_t)e[j] << LG)));
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (k0 + j >= ve) break;
                    const uint32_t mw[4] = {m[j].x, m[j].y, m[j].z, m[j].w};
                    for (int w = 0; w < 4; ++w) {
                        acc[2 * w] = vadd_16(acc[2 * w], prmt(mw[w], 0u, 0x9180u));
                        acc[2 * w + 1] = vadd_16(acc[2 * w + 1], prmt(mw[w], 0u, 0xB3A2u));
                    }
                }
            }
            uint4 *dst = reinterpret_cast<uint4 *>(L + pv);
            if (upd != 0xffffu) {
                // frames not updated keep their posterior
                const uint4 o0 = reinterpret_cast<const uint4 *>(Lc + pv)[0], o1 = reinterpret_cast<const uint4 *>(Lc + pv)[1];
                const uint32_t old[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
                for (int r = 0; r < 8; ++r) {
                    const uint32_t keep = (((upd >> (2 * r)) & 1u) ? 0u : 0x0000ffffu) |
                                          (((upd >> (2 * r + 1)) & 1u) ? 0u : 0xffff0000u);
                    acc[r] = (acc[r] & ~keep) | (old[r] & keep);
                }
            }
            dst[0] = make_uint4(acc[0], acc[1], acc[2], acc[3]);
            dst[1] = make_uint4(acc[4], acc[5], acc[6], acc[7]);
        }
    }
    prof_add(a.prof, units, bytes);
}

// Float-posterior flooding, variable side, 8 frames per thread: thread (listed
// frame block on y, (variable, group of 8 frames) on x) on a layout of 2^LG-frame
// blocks.  The same sums, in the same (ascending edge) order, as var_flood
// (FP32 accumulation of FP32 or FP16 messages); the edge indices of a chunk of
// four edges are loaded together, then their messages, so a variable of degree
// 3 is one round trip of index loads and one of message loads.
template <typename MsgT, int LG>
__global__ void __launch_bounds__(256) var_flood_x8(DecArgs a) {
    constexpr int G = (1 << LG) / 8;                   // groups of 8 frames per block
    const int64_t items = (int64_t)a.n * G;
    float *L = reinterpret_cast<float *>(a.L);
    const float *llr = reinterpret_cast<const float *>(a.llr_i);
    const MsgT *msg = reinterpret_cast<const MsgT *>(a.msg);
    unsigned long long units = 0, bytes = 0;
    const int32_t nblk = *a.blk_n;
    for (int32_t bi = blockIdx.y; bi < nblk; bi += gridDim.y) {
        const int64_t fb = __ldg(a.blk + bi);
        for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < items;
             idx += (int64_t)gridDim.x * blockDim.x) {
            const int64_t v = idx / G, f0 = (fb << LG) + ((idx % G) << 3);
            const int64_t bL = fpos(0, a.n, f0, LG), bM = fpos(0, a.E, f0, LG);
            if (v == 0 && (f0 & 31) == 0 && a.early_stop) a.unsat_next[f0 >> 5] = 0;   // next test starts clear
            const uint2 aw = *reinterpret_cast<const uint2 *>(a.active + f0);
            const uint32_t act = active_bits<4>(reinterpret_cast<const uint8_t *>(&aw.x)) |
                                 (active_bits<4>(reinterpret_cast<const uint8_t *>(&aw.y)) << 4);
            if (!act) continue;
            const uint32_t u = a.early_stop ? (__ldcg(a.unsat_cur + (f0 >> 5)) >> (f0 & 31)) & 0xffu : 0xffu;
            const uint32_t done = a.early_stop ? (act & ~u) : 0u;
            const uint32_t upd = act & ~done;
            if (v == 0)
                for (uint32_t r = done; r; r &= r - 1) {
                    const int i = __ffs(r) - 1;
                    a.active[f0 + i] = 0;
                    a.iters_i[f0 + i] = a.t - 1;
                }
            if (!upd) continue;
            const int32_t vb = __ldg(a.vptr + v), ve = __ldg(a.vptr + v + 1);
            const int64_t pv = bL + (v << LG);
            const unsigned nu = __popc(upd);
            units += nu;
            bytes += (unsigned long long)nu * ((ve - vb) * sizeof(MsgT) + 4 + 4);
            float acc[8];
            {
                const float4 c0 = __ldg(reinterpret_cast<const float4 *>(llr + pv));
                const float4 c1 = __ldg(reinterpret_cast<const float4 *>(llr + pv) + 1);
                acc[0] = c0.x; acc[1] = c0.y; acc[2] = c0.z; acc[3] = c0.w;
                acc[4] = c1.x; acc[5] = c1.y; acc[6] = c1.z; acc[7] = c1.w;
            }
            for (int32_t k0 = vb; k0 < ve; k0 += 4) {
                int32_t e[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) e[j] = __ldg(a.vedge + min(k0 + j, ve - 1));
                float m[4][8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (k0 + j >= ve) break;
                    const MsgT *mp = msg + bM + ((int64_t)e[j] << LG);
                    if (sizeof(MsgT) == 2) {
                        const uint4 h = __ldcs(reinterpret_cast<const uint4 *>(mp));
                        const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
                        for (int w = 0; w < 4; ++w) {
                            const float2 t = __half22float2(*reinterpret_cast<const __half2 *>(&hw[w]));
                            m[j][2 * w] = t.x;
                            m[j][2 * w + 1] = t.y;
                        }
                    } else {
                        const float4 m0 = __ldcs(reinterpret_cast<const float4 *>(mp));
                        const float4 m1 = __ldcs(reinterpret_cast<const float4 *>(mp) + 1);
                        m[j][0] = m0.x; m[j][1] = m0.y; m[j][2] = m0.z; m[j][3] = m0.w;
                        m[j][4] = m1.x; m[j][5] = m1.y; m[j][6] = m1.z; m[j][7] = m1.w;
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (k0 + j >= ve) break;
                    for (int i = 0; i < 8; ++i) acc[i] += m[j][i];
                }
            }
            float4 *dst = reinterpret_cast<float4 *>(L + pv);
            if (upd != 0xffu) {
                // frames not updated keep their posterior
                const float4 o0 = dst[0], o1 = dst[1];
                const float old[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
                for (int i = 0; i < 8; ++i)
                    if (!((upd >> i) & 1u)) acc[i] = old[i];
            }
            dst[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            dst[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        }
    }
    prof_add(a.prof, units, bytes);
}

// ------------------------------------------------------- layout conversions
// Frame placement of a decode pass: position f holds frame f, or, in a
// compacted re-decode, frame fmap[f] for f < *fcnt (the frames a first pass
// left unsatisfied, packed to the front; later positions hold no frame).
__device__ __forceinline__ int64_t frames_placed(int32_t F, const int32_t *fcnt) { return fcnt ? *fcnt : F; }
__device__ __forceinline__ int64_t frame_at(int64_t f, const int32_t *fmap) { return fmap ? fmap[f] : f; }

// llr [F][n] -> llr_i [n][Fp] and L [n][Fp]; padding frames get a
// confident all-zero word (they satisfy a zero syndrome at iteration 0).
template <int PREC>
__global__ void prep_llr(const float *__restrict__ llr, int32_t F, int32_t n, int64_t Fp, int lgfb,
                         float step, void *llr_i, void *L, const int32_t *fmap = nullptr,
                         const int32_t *fcnt = nullptr) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t v0 = (int64_t)blockIdx.x * 32;
    const int64_t Fv = frames_placed(F, fcnt);
    // positions past the placed frames of a compacted pass are never read
    const int64_t Fend = fcnt ? min(Fp, (Fv + 31) & ~(int64_t)31) : Fp;
    // frame groups of 32, grid-stride (a padded frame count can exceed 65535 groups)
    for (int64_t f0 = (int64_t)blockIdx.y * 32; f0 < Fend; f0 += (int64_t)gridDim.y * 32) {
    for (int r = 0; r < 32; r += 8) {
        const int64_t f = f0 + ty + r, v = v0 + tx;
        float val = kLlrClip;
        if (f < Fv && v < n) val = llr[frame_at(f, fmap) * n + v];
        tile[ty + r][tx] = val;
    }
    __syncthreads();
    for (int r = 0; r < 32; r += 8) {
        const int64_t v = v0 + ty + r, f = f0 + tx;
        if (v >= n || f >= Fp) continue;
        const float val = tile[tx][ty + r];
        const int64_t o = fpos(v, n, f, lgfb);
        if (PREC == kI8) {
            // round half away from zero on the step grid, clip to +-31
            const float rr = val / step;
            float q = floorf(fabsf(rr) + 0.5f);
            q = fminf(q, (float)kQMax);
            const int qi = (int)(rr < 0.0f ? -q : q);
            reinterpret_cast<int8_t *>(llr_i)[o] = (int8_t)qi;
            reinterpret_cast<int16_t *>(L)[o] = (int16_t)qi;
        } else {
            reinterpret_cast<float *>(llr_i)[o] = val;
            reinterpret_cast<float *>(L)[o] = val;
        }
    }
    __syncthreads();
    }
}

// synd [F][M] (bytes) -> sbits [M][W] (bit f%32 of word f/32).
__global__ void prep_synd(const uint8_t *__restrict__ synd, int32_t F, int32_t M, int64_t W,
                          uint32_t *__restrict__ sbits, const int32_t *fmap = nullptr,
                          const int32_t *fcnt = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t cbeg = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 64;
    const int64_t Fv = frames_placed(F, fcnt);
    const int64_t Wend = fcnt ? min(W, (Fv + 31) >> 5) : W;
    for (int64_t w = blockIdx.y; w < Wend; w += gridDim.y) {   // grid-stride over the words
        const int64_t f = w * 32 + lane;
        for (int64_t c = cbeg; c < cbeg + 64 && c < M; ++c) {
            const uint32_t bit = (f < Fv) ? (synd[frame_at(f, fmap) * M + c] & 1u) : 0u;
            const uint32_t word = __ballot_sync(0xffffffffu, bit);
            if (lane == 0) sbits[c * W + w] = word;
        }
    }
}

// packed syndromes [M][W_in] -> sbits [M][W] of this pass's layout (frames of
// a compacted pass gathered through fmap; positions past the placed frames 0)
__global__ void prep_synd_packed(const uint32_t *__restrict__ packed, int64_t W_in, int32_t F, int32_t M, int64_t W,
                                 uint32_t *__restrict__ sbits, const int32_t *fmap = nullptr,
                                 const int32_t *fcnt = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t cbeg = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 64;
    const int64_t Fv = frames_placed(F, fcnt);
    for (int64_t w = blockIdx.y; w < W; w += gridDim.y) {
        const int64_t f = w * 32 + lane;
        const int64_t g = f < Fv ? frame_at(f, fmap) : 0;
        for (int64_t c = cbeg; c < cbeg + 64 && c < M; ++c) {
            const uint32_t bit = (f < Fv) ? (__ldg(packed + c * W_in + (g >> 5)) >> (g & 31)) & 1u : 0u;
            const uint32_t word = __ballot_sync(0xffffffffu, bit);
            if (lane == 0) sbits[c * W + w] = word;
        }
    }
}

// per-frame state; `mask` marks the frames this decode owns (all real frames,
// or only the frames a low-precision pass left unsatisfied, in place or
// compacted to the first *fcnt positions)
__global__ void init_state(int32_t F, int64_t Fp, int64_t W, const uint8_t *__restrict__ conv_prev,
                           uint8_t *active, uint8_t *mask, int32_t *iters_i, uint32_t *unsat0,
                           uint32_t *unsat1, const int32_t *fcnt = nullptr) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f < W) {
        unsat0[f] = 0;
        unsat1[f] = 0;
    }
    if (f >= Fp) return;
    const uint8_t a = fcnt ? (f < *fcnt) : ((f < F) && (!conv_prev || !conv_prev[f]));
    active[f] = a;
    mask[f] = a;
    iters_i[f] = 0;
}

// `accumulate`: a re-decode adds its iterations to those of the first pass.
__global__ void finalize(int32_t F, int32_t T, int32_t accumulate, const uint8_t *__restrict__ mask,
                         const uint8_t *__restrict__ active, const int32_t *__restrict__ iters_i,
                         const uint32_t *__restrict__ unsat, int32_t *iters_out, uint8_t *conv_out,
                         const int32_t *fmap = nullptr) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F || !mask[f]) return;
    const int64_t g = frame_at(f, fmap);      // the frame at position f
    const int32_t base = accumulate ? iters_out[g] : 0;
    if (active[f]) {
        iters_out[g] = base + T;
        conv_out[g] = !((unsat[f >> 5] >> (f & 31)) & 1u);
    } else {
        iters_out[g] = base + iters_i[f];
        conv_out[g] = 1;
    }
}

// Compacted re-decode: the frames with conv_prev[f] == 0, packed to positions
// 0 .. *fcnt - 1 (*fcnt cleared before the launch).  Their order depends on
// scheduling; each frame decodes alone, so the results do not.
__global__ void compact_failed(int32_t F, const uint8_t *__restrict__ conv_prev, int32_t *fmap,
                               int32_t *fcnt) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool fail = f < F && !conv_prev[f];
    const uint32_t m = __ballot_sync(0xffffffffu, fail);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(fcnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (fail) fmap[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)f;
}

// Clear the messages of the frame blocks that hold placed frames (compacted
// pass: *fcnt frames from position 0; frame-block-major layout, so they are
// one contiguous prefix of block_bytes per block).
__global__ void zero_placed_msgs(uint4 *msg, int64_t block_bytes, int lgfb, const int32_t *fcnt) {
    const int64_t nb = ((int64_t)*fcnt + (1 << lgfb) - 1) >> lgfb;
    const int64_t words = nb * block_bytes / 16;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x)
        msg[i] = make_uint4(0u, 0u, 0u, 0u);
}

// L [n][Fp] -> bits [F][n] (+ posterior [F][n]) for the frames in `mask`.
template <int PREC>
__global__ void write_out(const void *Lp, int32_t F, int32_t n, int64_t Fp, int lgfb, float step,
                          const uint8_t *__restrict__ mask, uint8_t *bits, float *post,
                          const int32_t *fmap = nullptr, const int32_t *fcnt = nullptr) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t v0 = (int64_t)blockIdx.x * 32;
    const int64_t Fend = fcnt ? min(Fp, ((int64_t)*fcnt + 31) & ~(int64_t)31) : Fp;
    for (int64_t f0 = (int64_t)blockIdx.y * 32; f0 < Fend; f0 += (int64_t)gridDim.y * 32) {
    for (int r = 0; r < 32; r += 8) {
        const int64_t v = v0 + ty + r, f = f0 + tx;
        float val = 0.0f;
        if (v < n && f < Fp) {
            if (PREC == kI8) val = (float)reinterpret_cast<const int16_t *>(Lp)[fpos(v, n, f, lgfb)];
            else val = reinterpret_cast<const float *>(Lp)[fpos(v, n, f, lgfb)];
        }
        tile[tx][ty + r] = val;
    }
    __syncthreads();
    for (int r = 0; r < 32; r += 8) {
        const int64_t f = f0 + ty + r, v = v0 + tx;
        if (f >= F || v >= n || !mask[f]) continue;
        const float val = tile[ty + r][tx];
        const int64_t g = frame_at(f, fmap);
        bits[g * n + v] = val < 0.0f ? 1 : 0;
        if (post) post[g * n + v] = PREC == kI8 ? val * step : val;
    }
    __syncthreads();
    }
}

// ------------------------------------------------------------------ layout
struct Layout {
    int64_t Fp, FV, W;
    int lgfb;
    size_t llr_i, L, msg, sbits, active, mask, unsat0, unsat1, iters, blk, blk_n, fmap, fcnt, fsrc, total;
};

// register-cache size of the check kernels for a code: 8 or 32 edges, 0 = reload
static int dc_class(const CodeDev &d) { return d.dc_max <= 8 ? 8 : (d.dc_max <= kStash ? 32 : 0); }

// Frames per lane of the main kernel of a decode: one for sum-product and for
// the layered schedule (their per-edge state lives in registers), four for
// flooding min-sum.  The frame block is 32 lanes' worth of frames.
static int lanes_v(const CodeDev &d, int algo, int prec) {
    if (dc_class(d) == 0) return 4;
    if (algo == QKDREC_OMS_LAYERED) return 1;
    return (algo == QKDREC_SP_FLOOD && prec != kI8) ? 1 : 4;
}

static Layout make_layout(const CodeDev &d, int32_t F, int algo, int prec) {
    Layout l;
    l.lgfb = lanes_v(d, algo, prec) == 1 ? lgfb_of<1>() : lgfb_of<4>();
    l.Fp = align_up((size_t)(F > 0 ? F : 1), (size_t)1 << l.lgfb);
    l.FV = l.Fp / 4;
    l.W = ceil_div(l.Fp, 32);
    const size_t ms = prec == kF32 ? 4 : (prec == kF16 ? 2 : 1);
    const size_t ls = prec == kI8 ? 2 : 4;
    const size_t cs = prec == kI8 ? 1 : 4;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    l.llr_i = take((size_t)d.n * l.Fp * cs);
    l.L = take((size_t)d.n * l.Fp * ls);
    l.msg = take((size_t)d.E * l.Fp * ms);
    l.sbits = take((size_t)d.M * l.W * 4);
    l.active = take((size_t)l.Fp);
    l.mask = take((size_t)l.Fp);
    l.unsat0 = take((size_t)l.W * 4);
    l.unsat1 = take((size_t)l.W * 4);
    l.iters = take((size_t)l.Fp * 4);
    l.blk = take((size_t)(l.Fp >> l.lgfb) * 4);
    l.blk_n = take(4);
    l.fmap = take((size_t)l.Fp * 4);
    l.fcnt = take(4);
    l.fsrc = take((size_t)l.Fp * 4);
    l.total = off;
    return l;
}

// Iterations after which a flooding pass with the stopping test re-packs
// its still-decoding frames densely into the other half of its workspace (the
// frame blocks then hold only decoding frames again).  A fixed schedule, so the
// host always knows which half is live and the launches need no device
// decision; chosen on the measured iteration counts of the block-size sweep,
// where it lifts the decoding frames' share of the frame-block work from 0.75 to
// 0.87 after paying for the moves.
constexpr int kCompactAt[] = {16, 32, 64};
static bool compacts(const qkdrec_decode_opts &o, int algo, int prec) {
    (void)prec;
    return o.early_stop && algo != QKDREC_OMS_LAYERED && o.max_iter > kCompactAt[0];
}

static bool opts_ok(const qkdrec_decode_opts *o) {
    return o && o->algo >= 0 && o->algo <= 2 && o->prec >= 0 && o->prec <= 2 && o->max_iter >= 0 &&
           isfinite(o->offset) && o->offset >= 0.0f && isfinite(o->llr_step) && o->llr_step > 0.0f &&
           o->fallback_f32 >= 0 && o->fallback_f32 <= 2;
}

static size_t workspace_for(const CodeDev &d, int32_t F, const qkdrec_decode_opts *o) {
    size_t b = make_layout(d, F, o->algo, o->prec).total * (compacts(*o, o->algo, o->prec) ? 2 : 1);
    if (o->fallback_f32 && o->prec != kF32) {
        const int algo = o->fallback_f32 == 2 ? QKDREC_SP_FLOOD : o->algo;
        size_t b32 = make_layout(d, F, algo, kF32).total;   // the re-decode pass does not re-pack
        if (b32 > b) b = b32;
    }
    return b;
}

struct Prepared {
    uint32_t *unsat[2];
    uint8_t *mask;
};

// Launch geometry of a check-type kernel with V frames per lane.
struct Geom {
    dim3 grid;
    int fvw;
};
// The frame-block dimension of a kernel that walks the block list: enough CTAs
// to fill the device several times over; they stride over the listed blocks.
static Geom list_geom(int64_t Fp, int V, int64_t checks);
static Geom check_geom(int64_t Fp, int V, int64_t checks) {
    Geom g;
    const int64_t nvec = Fp / V;
    g.fvw = 1;
    while (g.fvw < 32 && g.fvw < nvec) g.fvw <<= 1;
    const int64_t per_block = (int64_t)kCheckWarps * kChecksPerWarp * (32 / g.fvw);
    const int64_t fblocks = ceil_div(nvec, g.fvw);
    g.grid = dim3((unsigned)ceil_div(checks, per_block), (unsigned)(fblocks < 65535 ? fblocks : 65535));
    return g;
}

static Geom list_geom(int64_t Fp, int V, int64_t checks) {
    Geom g = check_geom(Fp, V, checks);
    const int64_t target = (int64_t)sm_count() * 24;
    const int64_t gy = std::max<int64_t>(1, ceil_div(target, (int64_t)g.grid.x));
    if ((int64_t)g.grid.y > gy) g.grid.y = (unsigned)gy;
    return g;
}

// Frame blocks that still hold a decoding frame -> a.blk / a.blk_n (order of
// the list is the order blocks are found in; each block is processed the same
// way wherever it sits in the list).
__global__ void build_blocks(const uint8_t *__restrict__ active, int64_t nblk, int lgfb, int32_t *blk,
                             int32_t *blk_n) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool any = false;
    if (b < nblk) {
        const uint32_t *w = reinterpret_cast<const uint32_t *>(active + (b << lgfb));
        for (int k = 0; k < (1 << (lgfb - 2)); ++k) any |= w[k] != 0u;
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, any);
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && bal) base = atomicAdd(blk_n, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (any) blk[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)b;
}

static qkdrec_status rebuild_blocks(const Layout &l, char *ws, cudaStream_t st) {
    const int64_t nblk = l.Fp >> l.lgfb;
    int32_t *cnt = reinterpret_cast<int32_t *>(ws + l.blk_n);
    QKD_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t), st));
    build_blocks<<<(unsigned)ceil_div(nblk, 256), 256, 0, st>>>(
        reinterpret_cast<const uint8_t *>(ws + l.active), nblk, l.lgfb, reinterpret_cast<int32_t *>(ws + l.blk), cnt);
    QKD_LAUNCHED("build_blocks");
    return QKDREC_OK;
}

// The per-frame arrays of DecArgs and Prepared in the workspace half at ws.
static void bind(DecArgs &a, Prepared &pr, char *ws, const Layout &l) {
    a.sbits = reinterpret_cast<const uint32_t *>(ws + l.sbits);
    a.active = reinterpret_cast<uint8_t *>(ws + l.active);
    a.iters_i = reinterpret_cast<int32_t *>(ws + l.iters);
    a.L = ws + l.L;
    a.msg = ws + l.msg;
    a.llr_i = ws + l.llr_i;
    a.blk = reinterpret_cast<const int32_t *>(ws + l.blk);
    a.blk_n = reinterpret_cast<const int32_t *>(ws + l.blk_n);
    pr.unsat[0] = reinterpret_cast<uint32_t *>(ws + l.unsat0);
    pr.unsat[1] = reinterpret_cast<uint32_t *>(ws + l.unsat1);
    pr.mask = reinterpret_cast<uint8_t *>(ws + l.mask);
}

// ------------------------------------------------------ frame re-packing
// rmask = frames of this half that have stopped (their outputs are final)
__global__ void retired_mask(int64_t Fp, const uint8_t *__restrict__ mask, const uint8_t *__restrict__ active,
                             uint8_t *__restrict__ rmask) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < Fp; f += (int64_t)gridDim.x * blockDim.x)
        rmask[f] = mask[f] && !active[f];
}
// positions of the decoding frames, packed to fsrc[0 .. *cnt) (*cnt cleared
// before); a warp's frames keep their order, so consecutive new positions mostly
// come from one old frame block
__global__ void list_active(int64_t Fp, const uint8_t *__restrict__ active, int32_t *fsrc, int32_t *cnt) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = f < Fp && active[f];
    const uint32_t m = __ballot_sync(0xffffffffu, on);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(cnt, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (on) fsrc[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)f;
}
// new position p holds old position fsrc[p]: its frame is fmap_old[fsrc[p]]
__global__ void remap_frames(const int32_t *__restrict__ fsrc, const int32_t *__restrict__ cnt,
                             const int32_t *__restrict__ fmap_old, int32_t *__restrict__ fmap_new) {
    const int64_t c = *cnt;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < c; p += (int64_t)gridDim.x * blockDim.x)
        fmap_new[p] = fmap_old ? fmap_old[fsrc[p]] : fsrc[p];
}
// The values (32-, 16- or 8-bit) of every item (variable or edge) of the
// re-packed frames: one warp per (32 new positions, item), writes coalesced
template <typename T>
__global__ void gather_frames(const T *__restrict__ src, T *__restrict__ dst, int64_t items, int lgfb,
                              const int32_t *__restrict__ fsrc, const int32_t *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t c = *cnt, words = (c + 31) >> 5, tasks = words * items;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tasks; t += wstride) {
        const int64_t w = t / items, item = t - w * items, p = (w << 5) + lane;
        T v = 0;
        if (p < c) v = src[fpos(item, items, __ldg(fsrc + p), lgfb)];
        dst[fpos(item, items, p, lgfb)] = v;
    }
}
// per-frame state of the new half: positions < *cnt decoding
__global__ void init_repacked(int64_t Fp, int64_t W, const int32_t *__restrict__ cnt, uint8_t *active,
                              uint8_t *mask, int32_t *iters_i, uint32_t *unsat0, uint32_t *unsat1) {
    const int64_t c = *cnt;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < Fp; f += (int64_t)gridDim.x * blockDim.x) {
        active[f] = f < c;
        mask[f] = f < c;
        iters_i[f] = 0;
        if (f < W) {
            unsat0[f] = 0;
            unsat1[f] = 0;
        }
    }
}

// Shared set-up of one decode pass: per-frame state, interleaved LLRs and
// posteriors, packed syndromes, zero messages.
// compact: decode the frames with conv_prev[f] == 0 packed to the front (a
// re-decode then touches only the frame blocks that hold them)
static qkdrec_status prepare(const CodeDev &d, const float *llr, const SyndIn &synd, int32_t F,
                             const qkdrec_decode_opts &o, int prec, const uint8_t *conv_prev, bool compact,
                             char *ws, const Layout &l, cudaStream_t st, DecArgs &a, Prepared &pr) {
    a.rp = d.rp;
    a.ci = d.ci;
    a.vptr = d.vptr;
    a.vedge = d.vedge;
    bind(a, pr, ws, l);
    a.Fp = l.Fp;
    a.FV = l.FV;
    a.E = d.E;
    a.lgfb = l.lgfb;
    a.W = l.W;
    a.n = d.n;
    a.M = d.M;
    a.fvw = 32;
    a.dstash = kStash;
    a.t = 0;
    a.do_msgs = 1;
    a.early_stop = o.early_stop ? 1 : 0;
    a.beta = o.offset;
    a.prof = nullptr;
    a.unsat_cur = pr.unsat[0];
    a.unsat_next = pr.unsat[1];
    int32_t *fmap = compact ? reinterpret_cast<int32_t *>(ws + l.fmap) : nullptr;
    int32_t *fcnt = compact ? reinterpret_cast<int32_t *>(ws + l.fcnt) : nullptr;
    if (compact) {
        QKD_CUDA(cudaMemsetAsync(fcnt, 0, sizeof(int32_t), st));
        prof::Scope ps(prof::kPrep, st);
        compact_failed<<<(unsigned)ceil_div(F, 256), 256, 0, st>>>(F, conv_prev, fmap, fcnt);
        QKD_LAUNCHED("compact_failed");
    }
    {
        prof::Scope ps(prof::kPrep, st);
        init_state<<<(unsigned)ceil_div(std::max<int64_t>(l.Fp, l.W), 256), 256, 0, st>>>(
            F, l.Fp, l.W, conv_prev, a.active, pr.mask, a.iters_i, pr.unsat[0], pr.unsat[1], fcnt);
    }
    QKD_LAUNCHED("init_state");
    {
        prof::Scope ps(prof::kPrep, st);
        dim3 blk(32, 8), grd((unsigned)ceil_div(d.n, 32), (unsigned)std::min<int64_t>(ceil_div(l.Fp, 32), 65535));
        if (prec == kI8)
            prep_llr<kI8><<<grd, blk, 0, st>>>(llr, F, d.n, l.Fp, l.lgfb, o.llr_step, ws + l.llr_i, ws + l.L, fmap,
                                                fcnt);
        else prep_llr<kF32><<<grd, blk, 0, st>>>(llr, F, d.n, l.Fp, l.lgfb, o.llr_step, ws + l.llr_i, ws + l.L,
                                                  fmap, fcnt);
    }
    QKD_LAUNCHED("prep_llr");
    {
        prof::Scope ps(prof::kPrep, st);
        dim3 grd((unsigned)ceil_div(d.M, 8 * 64), (unsigned)std::min<int64_t>(l.W, 65535));
        if (synd.packed)
            prep_synd_packed<<<grd, 256, 0, st>>>(synd.packed, synd.W, F, d.M, l.W,
                                                  reinterpret_cast<uint32_t *>(ws + l.sbits), fmap, fcnt);
        else
            prep_synd<<<grd, 256, 0, st>>>(synd.bytes, F, d.M, l.W, reinterpret_cast<uint32_t *>(ws + l.sbits), fmap,
                                           fcnt);
    }
    QKD_LAUNCHED("prep_synd");
    const size_t ms = prec == kF32 ? 4 : (prec == kF16 ? 2 : 1);
    if (compact) {
        prof::Scope ps(prof::kPrep, st);
        zero_placed_msgs<<<(unsigned)sm_count() * 8, 256, 0, st>>>(reinterpret_cast<uint4 *>(ws + l.msg),
                                                                    (int64_t)d.E * ms << l.lgfb, l.lgfb, fcnt);
        QKD_LAUNCHED("zero_placed_msgs");
    } else {
        QKD_CUDA(cudaMemsetAsync(ws + l.msg, 0, (size_t)d.E * l.Fp * ms, st));
    }
    prof::Scope ps(prof::kPrep, st);
    return rebuild_blocks(l, ws, st);
}

// Shared tail: iteration counts / converged flags, then bits and posteriors
// back to the frame-major output layout.
static qkdrec_status finish(const CodeDev &d, int32_t F, int T, int prec, const qkdrec_decode_opts &o,
                            const uint8_t *conv_prev, const int32_t *fmap, const int32_t *fcnt, char *ws,
                            const Layout &l, const Prepared &pr, const DecArgs &a, int final_buf, uint8_t *bits_out,
                            int32_t *iters_out, uint8_t *conv_out, float *post_out, cudaStream_t st) {
    {
        prof::Scope ps(prof::kFinish, st);
        finalize<<<(unsigned)ceil_div(F, 256), 256, 0, st>>>(F, T, conv_prev ? 1 : 0, pr.mask, a.active,
                                                             a.iters_i, pr.unsat[final_buf], iters_out, conv_out,
                                                             fmap);
    }
    QKD_LAUNCHED("finalize");
    prof::Scope ps(prof::kFinish, st);
    dim3 blk(32, 8), grd((unsigned)ceil_div(d.n, 32), (unsigned)std::min<int64_t>(ceil_div(l.Fp, 32), 65535));
    if (prec == kI8)
        write_out<kI8><<<grd, blk, 0, st>>>(ws + l.L, F, d.n, l.Fp, l.lgfb, o.llr_step, pr.mask, bits_out, post_out,
                                            fmap, fcnt);
    else write_out<kF32><<<grd, blk, 0, st>>>(ws + l.L, F, d.n, l.Fp, l.lgfb, o.llr_step, pr.mask, bits_out,
                                              post_out, fmap, fcnt);
    QKD_LAUNCHED("write_out");
    return QKDREC_OK;
}

// Launch one flooding check kernel (or its parity-only form).  SP keeps one
// frame per lane so that the phi values of a check fit in registers; min-sum
// only keeps sign bits and runs four frames per lane.
// The kernels' frame block is fixed at compile time by V (lgfb_of), so V follows
// the layout of the decode: one frame per lane on 32-frame blocks (sum-product
// and layered schedules), four on 128-frame blocks (flooding min-sum).
static void launch_check(DecArgs a, const CodeDev &d, int algo, int prec, cudaStream_t st) {
    const bool cached = dc_class(d) > 0;
    const int V = a.lgfb == lgfb_of<1>() ? 1 : 4;
    const Geom g = list_geom(a.Fp, V, d.M);
    a.fvw = g.fvw;
    const dim3 B(kCheckWarps * 32);
    a.dstash = std::min(std::max(d.dc_max, 1), kStash);
    const size_t stash = (size_t)kCheckWarps * a.dstash * 32 * sizeof(float);
    if (prec == kI8) {
        // 16-bit lanes need L - m to stay inside int16: |L| <= kQMax (dv + 1)
        if (V == 1) check_flood_i<1, 32><<<g.grid, B, 0, st>>>(a);
        else if (cached && d.dv_max <= 1000)
            check_flood_i16x2<<<g.grid, B, (size_t)kCheckWarps * a.dstash * 32 * sizeof(uint32_t), st>>>(a);
        else if (cached) check_flood_i<4, 32><<<g.grid, B, 0, st>>>(a);
        else check_flood_i<4, 0><<<g.grid, B, 0, st>>>(a);
    } else if (algo == QKDREC_SP_FLOOD) {
        if (prec == kF32) {
            if (V == 1 && a.do_msgs && g.fvw == 32) {
                // two frames per lane, half-warps on two listed blocks
                const size_t stash2 = (size_t)kCheckWarps * a.dstash * 32 * sizeof(float2);
                static bool attr_set[64] = {false};   // per device
                int dev = 0;
                cudaGetDevice(&dev);
                if (dev >= 0 && dev < 64 && !attr_set[dev]) {
                    cudaFuncSetAttribute(check_flood_sp2<kSp2Chunk>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((size_t)kCheckWarps * kStash * 32 * sizeof(float2)));
                    attr_set[dev] = true;
                }
                dim3 g2 = g.grid;
                g2.y = (g2.y + 1) / 2;
                check_flood_sp2<kSp2Chunk><<<g2, B, stash2, st>>>(a);
            } else if (V == 1) check_flood_f<kSP, float, 1, true><<<g.grid, B, stash, st>>>(a);
            else check_flood_f<kSP, float, 4, false><<<g.grid, B, 0, st>>>(a);
        } else {
            if (V == 1) check_flood_f<kSP, __half, 1, true><<<g.grid, B, stash, st>>>(a);
            else check_flood_f<kSP, __half, 4, false><<<g.grid, B, 0, st>>>(a);
        }
    } else {
        if (prec == kF32) {
            if (V == 1) check_flood_f<kOMS, float, 1, true><<<g.grid, B, 0, st>>>(a);
            else if (cached) check_flood_f<kOMS, float, 4, true><<<g.grid, B, 0, st>>>(a);
            else check_flood_f<kOMS, float, 4, false><<<g.grid, B, 0, st>>>(a);
        } else {
            if (V == 1) check_flood_f<kOMS, __half, 1, true><<<g.grid, B, 0, st>>>(a);
            else if (cached) check_flood_f<kOMS, __half, 4, true><<<g.grid, B, 0, st>>>(a);
            else check_flood_f<kOMS, __half, 4, false><<<g.grid, B, 0, st>>>(a);
        }
    }
}

// One flooding decode pass over the frames selected by conv_prev (NULL = all).
static qkdrec_status run_flood(const CodeDev &d, const float *llr, const SyndIn &synd, int32_t F,
                               const qkdrec_decode_opts &o, int prec, const uint8_t *conv_prev, bool compact,
                               uint8_t *bits_out, int32_t *iters_out, uint8_t *conv_out,
                               float *post_out, char *ws, cudaStream_t st) {
    const Layout l = make_layout(d, F, o.algo, prec);
    DecArgs a;
    Prepared pr;
    qkdrec_status s = prepare(d, llr, synd, F, o, prec, conv_prev, compact, ws, l, st, a, pr);
    if (s != QKDREC_OK) return s;
    // the live workspace half and its frame placement (NULL: position = frame)
    char *cur = ws;
    const int32_t *fmap_cur = compact ? reinterpret_cast<const int32_t *>(ws + l.fmap) : nullptr;
    const int32_t *fcnt_cur = compact ? reinterpret_cast<const int32_t *>(ws + l.fcnt) : nullptr;
    // a re-decode pass holds only frames a first pass could not solve, which
    // mostly run every iteration: re-packing them would move them for nothing
    const bool repack = compacts(o, o.algo, prec) && !compact;
    const int64_t vitems = (int64_t)d.n * l.FV;
    const unsigned vgrid = (unsigned)std::min<int64_t>(ceil_div(vitems, 256), (int64_t)sm_count() * 64);
    // integer form: (variable, 16 frames) on x, listed frame blocks on y; FP16
    // messages: (variable, 8 frames)
    const bool i16 = prec == kI8 && l.lgfb == lgfb_of<4>() && d.dv_max <= 1000;
    const bool x8 = prec != kI8;     // 8 frames per thread, 32- or 128-frame blocks
    const int groups = x8 ? (1 << l.lgfb) / 8 : 8;
    dim3 igrid((unsigned)std::min<int64_t>(ceil_div((int64_t)d.n * groups, 256), (int64_t)sm_count() * 64), 1);
    igrid.y = (unsigned)std::max<int64_t>(1, std::min<int64_t>(l.Fp >> l.lgfb, (int64_t)sm_count() * 64 / igrid.x));

    auto check = [&](int t, int do_msgs) {
        a.t = t;
        a.do_msgs = do_msgs;
        a.unsat_cur = pr.unsat[t & 1];
        a.unsat_next = pr.unsat[(t + 1) & 1];
        const int kind = !do_msgs ? (prec == kI8 ? prof::kParityI8 : prof::kParityF32)
                         : prec == kI8 ? prof::kCheckOmsI8
                         : o.algo == QKDREC_SP_FLOOD ? (prec == kF32 ? prof::kCheckSpF32 : prof::kCheckSpF16)
                                                     : (prec == kF32 ? prof::kCheckOmsF32 : prof::kCheckOmsF16);
        a.prof = prof::counters(kind);
        prof::Scope ps(kind, st);
        launch_check(a, d, o.algo, prec, st);
    };
    for (int t = 1; t <= o.max_iter; ++t) {
        check(t, 1);
        QKD_LAUNCHED("check_flood");
        a.t = t;
        {
            const int kind = prec == kI8 ? prof::kVarI8 : (prec == kF16 ? prof::kVarF16 : prof::kVarF32);
            a.prof = prof::counters(kind);
            prof::Scope ps(kind, st);
            if (i16) var_flood_i8x16<<<igrid, 256, 0, st>>>(a);
            else if (prec == kI8) var_flood<kI8><<<vgrid, 256, 0, st>>>(a);
            else if (l.lgfb == lgfb_of<1>()) {
                if (prec == kF16) var_flood_x8<__half, lgfb_of<1>()><<<igrid, 256, 0, st>>>(a);
                else var_flood_x8<float, lgfb_of<1>()><<<igrid, 256, 0, st>>>(a);
            } else {
                if (prec == kF16) var_flood_x8<__half, lgfb_of<4>()><<<igrid, 256, 0, st>>>(a);
                else var_flood_x8<float, lgfb_of<4>()><<<igrid, 256, 0, st>>>(a);
            }
        }
        QKD_LAUNCHED("var_flood");
        if (o.early_stop) {
            // frames retired by this variable pass leave the list
            prof::Scope ps(prof::kFinish, st);
            if ((s = rebuild_blocks(l, cur, st)) != QKDREC_OK) return s;
        }
        if (repack && t < o.max_iter && std::find(std::begin(kCompactAt), std::end(kCompactAt), t) != std::end(kCompactAt)) {
            // the frames that stopped leave with their final outputs; the decoding
            // ones move, state and all, to the front of the other half
            prof::Scope ps(prof::kRepack, st);
            char *nxt = cur == ws ? ws + l.total : ws;
            uint8_t *rmask = reinterpret_cast<uint8_t *>(nxt + l.mask);
            const unsigned gF = (unsigned)std::min<int64_t>(ceil_div(l.Fp, 256), (int64_t)sm_count() * 32);
            retired_mask<<<gF, 256, 0, st>>>(l.Fp, pr.mask, a.active, rmask);
            finalize<<<(unsigned)ceil_div(F, 256), 256, 0, st>>>(F, t, conv_prev ? 1 : 0, rmask, a.active, a.iters_i,
                                                                 pr.unsat[0], iters_out, conv_out, fmap_cur);
            {
                dim3 blk(32, 8), grd((unsigned)ceil_div(d.n, 32), (unsigned)std::min<int64_t>(ceil_div(l.Fp, 32), 65535));
                if (prec == kI8)
                    write_out<kI8><<<grd, blk, 0, st>>>(a.L, F, d.n, l.Fp, l.lgfb, o.llr_step, rmask, bits_out,
                                                        post_out, fmap_cur, fcnt_cur);
                else
                    write_out<kF32><<<grd, blk, 0, st>>>(a.L, F, d.n, l.Fp, l.lgfb, o.llr_step, rmask, bits_out,
                                                         post_out, fmap_cur, fcnt_cur);
            }
            int32_t *fsrc = reinterpret_cast<int32_t *>(nxt + l.fsrc), *fcnt_n = reinterpret_cast<int32_t *>(nxt + l.fcnt);
            int32_t *fmap_n = reinterpret_cast<int32_t *>(nxt + l.fmap);
            QKD_CUDA(cudaMemsetAsync(fcnt_n, 0, sizeof(int32_t), st));
            list_active<<<(unsigned)ceil_div(l.Fp, 256), 256, 0, st>>>(l.Fp, a.active, fsrc, fcnt_n);
            remap_frames<<<gF, 256, 0, st>>>(fsrc, fcnt_n, fmap_cur, fmap_n);
            const unsigned gG = (unsigned)sm_count() * 16;
            // element sizes of the layout: channel values, posteriors, messages
            auto gather = [&](size_t off, int64_t items, int bytes) {
                if (bytes == 4)
                    gather_frames<uint32_t><<<gG, 256, 0, st>>>(reinterpret_cast<const uint32_t *>(cur + off),
                                                                reinterpret_cast<uint32_t *>(nxt + off), items,
                                                                l.lgfb, fsrc, fcnt_n);
                else if (bytes == 2)
                    gather_frames<uint16_t><<<gG, 256, 0, st>>>(reinterpret_cast<const uint16_t *>(cur + off),
                                                                reinterpret_cast<uint16_t *>(nxt + off), items,
                                                                l.lgfb, fsrc, fcnt_n);
                else
                    gather_frames<uint8_t><<<gG, 256, 0, st>>>(reinterpret_cast<const uint8_t *>(cur + off),
                                                               reinterpret_cast<uint8_t *>(nxt + off), items, l.lgfb,
                                                               fsrc, fcnt_n);
            };
            gather(l.llr_i, d.n, prec == kI8 ? 1 : 4);
            gather(l.L, d.n, prec == kI8 ? 2 : 4);
            gather(l.msg, d.E, prec == kF32 ? 4 : (prec == kF16 ? 2 : 1));
            {
                dim3 grd((unsigned)ceil_div(d.M, 8 * 64), (unsigned)std::min<int64_t>(l.W, 65535));
                prep_synd_packed<<<grd, 256, 0, st>>>(a.sbits, l.W, F, d.M, l.W,
                                                      reinterpret_cast<uint32_t *>(nxt + l.sbits), fsrc, fcnt_n);
            }
            Prepared pn;
            bind(a, pn, nxt, l);
            init_repacked<<<gF, 256, 0, st>>>(l.Fp, l.W, fcnt_n, a.active, pn.mask, a.iters_i, pn.unsat[0], pn.unsat[1]);
            QKD_LAUNCHED("frame re-packing");
            pr = pn;
            cur = nxt;
            fmap_cur = fmap_n;
            fcnt_cur = fcnt_n;
            if ((s = rebuild_blocks(l, cur, st)) != QKDREC_OK) return s;
        }
    }
    // stopping test on the final posteriors (parity buffer (T+1)&1 is clear)
    const int T = o.max_iter;
    a.early_stop = 1;
    check(T + 1, 0);
    QKD_LAUNCHED("check_flood(parity)");
    return finish(d, F, T, prec, o, conv_prev, fmap_cur, fcnt_cur, cur, l, pr, a, (T + 1) & 1, bits_out, iters_out,
                  conv_out, post_out, st);
}

#include "decode_layered.cuh"

__global__ void phi_selftest_kernel(const float *__restrict__ x, int64_t count, float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = phi_clamped(x[i]);
}
// phi2 on consecutive pairs, clamped as the two-frame kernel clamps |q|
__global__ void phi_pair_selftest_kernel(const float *__restrict__ x, int64_t pairs, float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pairs; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = reinterpret_cast<const float2 *>(x)[i];
        reinterpret_cast<float2 *>(out)[i] = phi2(make_float2(fmaxf(fminf(fabsf(v.x), kAMax), kAMin),
                                                              fmaxf(fminf(fabsf(v.y), kAMax), kAMin)));
    }
}

qkdrec_status decode_batch_impl(qkdrec_code_t code, const float *llr, const SyndIn &synd, int32_t F,
                                const qkdrec_decode_opts *opts, uint8_t *bits_out, int32_t *iters_out,
                                uint8_t *conv_out, float *post_out, void *workspace, size_t workspace_bytes,
                                void *stream) {
    clear_error();
    if (!code) QKD_FAIL(QKDREC_ERR_ARG, "code is NULL");
    if (F < 0) QKD_FAIL(QKDREC_ERR_ARG, "F < 0");
    if (!opts_ok(opts)) QKD_FAIL(QKDREC_ERR_ARG, "bad decode options");
    const qkdrec_decode_opts o = *opts;
    if (o.prec == QKDREC_I8SAT && o.algo == QKDREC_SP_FLOOD)
        QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "integer messages need an offset min-sum algorithm");
    if (F == 0) return QKDREC_OK;
    if (F > kMaxFrames) QKD_FAIL(QKDREC_ERR_ARG, "F=%d above the %d frames of one launch", F, kMaxFrames);
    if (!llr || !(synd.bytes || synd.packed) || !bits_out || !iters_out || !conv_out)
        QKD_FAIL(QKDREC_ERR_ARG, "NULL input/output");
    if (synd.packed && synd.W < ceil_div(F, 32)) QKD_FAIL(QKDREC_ERR_ARG, "packed syndrome rows too short");
    if (!workspace) QKD_FAIL(QKDREC_ERR_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) % 256) QKD_FAIL(QKDREC_ERR_ARG, "workspace not 256-byte aligned");
    const size_t need = workspace_for(code->d, F, &o);
    if (workspace_bytes < need) QKD_FAIL(QKDREC_ERR_ARG, "workspace %zu bytes < %zu needed", workspace_bytes, need);
    const CodeDev &d = code->d;
    cudaStream_t st = as_stream(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    qkdrec_status s;
    auto pass = [&](const qkdrec_decode_opts &po, int prec, const uint8_t *conv_prev, bool compact) {
        if (po.algo == QKDREC_OMS_LAYERED)
            return run_layered(d, llr, synd, F, po, prec, conv_prev, compact, bits_out, iters_out, conv_out,
                               post_out, ws, st);
        return run_flood(d, llr, synd, F, po, prec, conv_prev, compact, bits_out, iters_out, conv_out, post_out,
                         ws, st);
    };
    if ((s = pass(o, o.prec, nullptr, false)) != QKDREC_OK) return s;
    // FP32 re-decode of the frames a low-precision pass left unsatisfied,
    // compacted to the front so that it costs what the failed frames need
    if (o.fallback_f32 && o.prec != QKDREC_F32) {
        qkdrec_decode_opts o2 = o;
        if (o.fallback_f32 == 2) o2.algo = QKDREC_SP_FLOOD;
        if ((s = pass(o2, QKDREC_F32, conv_out, true)) != QKDREC_OK) return s;
    }
    return QKDREC_OK;
}

}  // namespace qkd

using namespace qkd;

extern "C" {

qkdrec_status qkdrec_selftest_phi(const float *x, int64_t count, float *out, void *stream) {
    clear_error();
    if (count < 0) QKD_FAIL(QKDREC_ERR_ARG, "count < 0");
    if (count == 0) return QKDREC_OK;
    if (!x || !out) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    phi_selftest_kernel<<<(unsigned)std::min<int64_t>(ceil_div(count, 256), 4096), 256, 0, as_stream(stream)>>>(
        x, count, out);
    QKD_LAUNCHED("phi_selftest_kernel");
    return QKDREC_OK;
}

qkdrec_status qkdrec_selftest_phi_pair(const float *x, int64_t count, float *out, void *stream) {
    clear_error();
    if (count < 0 || count % 2) QKD_FAIL(QKDREC_ERR_ARG, "count must be even and >= 0");
    if (count == 0) return QKDREC_OK;
    if (!x || !out) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    if (reinterpret_cast<uintptr_t>(x) % 8 || reinterpret_cast<uintptr_t>(out) % 8)
        QKD_FAIL(QKDREC_ERR_ARG, "x/out must be 8-byte aligned");
    phi_pair_selftest_kernel<<<(unsigned)std::min<int64_t>(ceil_div(count / 2, 256), 4096), 256, 0,
                               as_stream(stream)>>>(x, count / 2, out);
    QKD_LAUNCHED("phi_pair_selftest_kernel");
    return QKDREC_OK;
}

void qkdrec_decode_opts_default(qkdrec_decode_opts *o) {
    if (!o) return;
    o->algo = QKDREC_SP_FLOOD;
    o->prec = QKDREC_F32;
    o->max_iter = 50;
    o->offset = 0.5f;
    o->llr_step = 0.5f;
    o->early_stop = 1;
    o->fallback_f32 = 0;
}

qkdrec_status qkdrec_decode_workspace_size(qkdrec_code_t code, int32_t F, const qkdrec_decode_opts *opts,
                                           size_t *bytes) {
    clear_error();
    if (!code || !bytes) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    if (F < 0) QKD_FAIL(QKDREC_ERR_ARG, "F < 0");
    if (!opts_ok(opts)) QKD_FAIL(QKDREC_ERR_ARG, "bad decode options");
    *bytes = workspace_for(code->d, F, opts);
    return QKDREC_OK;
}

qkdrec_status qkdrec_decode_batch(qkdrec_code_t code, const float *llr, const uint8_t *synd, int32_t F,
                                  const qkdrec_decode_opts *opts, uint8_t *bits_out, int32_t *iters_out,
                                  uint8_t *conv_out, float *post_out, void *workspace,
                                  size_t workspace_bytes, void *stream) {
    SyndIn si;
    si.bytes = synd;
    return decode_batch_impl(code, llr, si, F, opts, bits_out, iters_out, conv_out, post_out, workspace,
                             workspace_bytes, stream);
}

}  // extern "C"

extern "C" qkdrec_status qkdrec_qc_timeouts(int32_t *count) {
    clear_error();
    if (!count) QKD_FAIL(QKDREC_ERR_ARG, "count is NULL");
    QKD_CUDA(cudaMemcpyFromSymbol(count, qkd::g_qc_timeouts, sizeof(int32_t)));
    return QKDREC_OK;
}

#include "decode_woms.cuh"
#include "decode_plan.cuh"

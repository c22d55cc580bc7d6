// Syndrome-based BP decoding of many sub-blocks sharing one parity-check matrix
// (Sec. III-A: N_d decoders loaded with the same matrix; Sec. III-C: BP decoder).
//
// Data layout (frame-interleaved): every per-variable or per-edge quantity is
// stored as [item][Fp] with the frame index fastest, Fp = F rounded up to a
// multiple of 4.  A lane owns a "frame vector" of 4 consecutive frames, so each
// access is a 16-byte (FP32), 8-byte (FP16) or 4-byte (int8) vector and a warp
// touches one contiguous run per edge: the column index of an edge is loaded
// once and reused by all frames.
//
//   llr_i [n][Fp]   channel LLR (float; int8 on the 6-bit grid in integer mode)
//   L     [n][Fp]   posterior (float; int16 in integer mode)
//   msg   [E][Fp]   check-to-variable messages in CSR edge order (float/half/int8)
//   sbits [M][W]    syndrome bits, 32 frames per word
//   active[Fp]      1 while the frame is decoding
//   unsat [2][Fp/4] per frame vector: bit i set if frame 4fv+i had an
//                   unsatisfied check (double-buffered by iteration parity)
//
// One iteration = check kernel + variable kernel.  The check kernel of
// iteration t reads L^(t-1) for every edge anyway, so it also forms the parity
// of the hard decision of L^(t-1) on every check: that is the stopping test of
// the previous iteration, at no extra traffic.  The variable kernel of
// iteration t then retires frames whose test passed (iters = t-1, posterior
// frozen) and updates the others.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "profile.cuh"

namespace qkd {

enum Prec { kF32 = 0, kF16 = 1, kI8 = 2 };
enum Algo { kSP = 0, kOMS = 1 };

constexpr int kCheckWarps = 8;   // warps per check-kernel block
constexpr int kChecksPerWarp = 4;
constexpr int32_t kMaxFrames = 65535 * 32;  // syndrome packing uses one grid row per 32 frames

// ---------------------------------------------------------------- vector I/O
struct F4 { float v[4]; };

__device__ __forceinline__ F4 ld_f4(const float *p) {
    float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    return F4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ void st_f4(float *p, const F4 &a) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
__device__ __forceinline__ F4 ld_msg(const float *p) { return ld_f4(p); }
__device__ __forceinline__ void st_msg(float *p, const F4 &a) { st_f4(p, a); }
__device__ __forceinline__ F4 ld_msg(const __half *p) {
    uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
    __half2 a = *reinterpret_cast<__half2 *>(&t.x), b = *reinterpret_cast<__half2 *>(&t.y);
    float2 fa = __half22float2(a), fb = __half22float2(b);
    return F4{{fa.x, fa.y, fb.x, fb.y}};
}
__device__ __forceinline__ void st_msg(__half *p, const F4 &a) {
    __half2 x = __floats2half2_rn(a.v[0], a.v[1]), y = __floats2half2_rn(a.v[2], a.v[3]);
    uint2 t;
    t.x = *reinterpret_cast<uint32_t *>(&x);
    t.y = *reinterpret_cast<uint32_t *>(&y);
    *reinterpret_cast<uint2 *>(p) = t;
}

// value a message has after being stored (FP16 rounding, identity for FP32)
template <typename MsgT> __device__ __forceinline__ F4 as_stored(const F4 &a);
template <> __device__ __forceinline__ F4 as_stored<float>(const F4 &a) { return a; }
template <> __device__ __forceinline__ F4 as_stored<__half>(const F4 &a) {
    F4 r;
    for (int i = 0; i < 4; ++i) r.v[i] = __half2float(__float2half_rn(a.v[i]));
    return r;
}

struct I4 { int v[4]; };
__device__ __forceinline__ I4 ld_i8x4(const int8_t *p) {
    char4 t = __ldg(reinterpret_cast<const char4 *>(p));
    return I4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ void st_i8x4(int8_t *p, const I4 &a) {
    *reinterpret_cast<char4 *>(p) = make_char4((signed char)a.v[0], (signed char)a.v[1],
                                                (signed char)a.v[2], (signed char)a.v[3]);
}
__device__ __forceinline__ I4 ld_i16x4(const int16_t *p) {
    short4 t = __ldg(reinterpret_cast<const short4 *>(p));
    return I4{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ void st_i16x4(int16_t *p, const I4 &a) {
    *reinterpret_cast<short4 *>(p) = make_short4((short)a.v[0], (short)a.v[1], (short)a.v[2], (short)a.v[3]);
}

// phi(x) = -ln tanh(x/2) = ln((e^x + 1)/(e^x - 1)), evaluated as log1p(2 / expm1(x));
// it is its own inverse on (0, inf).
__device__ __forceinline__ float phi_f(float x) { return log1pf(2.0f / expm1f(x)); }

__device__ __forceinline__ uint32_t active4(const uint8_t *active, int64_t fv) {
    return *reinterpret_cast<const uint32_t *>(active + 4 * fv);  // byte i = frame 4fv+i
}
__device__ __forceinline__ bool act_bit(uint32_t a4, int i) { return (a4 >> (8 * i)) & 0xff; }

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
    int64_t FV, W;
    int32_t n, M;
    int32_t fvw;            // frame vectors per warp row (power of two <= 32)
    int32_t t;              // iteration index (1-based)
    int32_t early_stop;
    int32_t do_msgs;        // 0: parity test only
    float beta;             // OMS offset (float modes)
    unsigned long long *prof;  // (units, bytes) counters of this launch's kernel class, or NULL
};

// Reduce 4-bit unsatisfied masks of the lanes that own the same frame vector,
// across the warp and the block, then publish them with one atomic per vector.
__device__ __forceinline__ void publish_unsat(uint32_t bits, int fvw, int lane, int warp,
                                              int64_t fv, bool fv_ok, uint32_t *unsat) {
    __shared__ uint32_t blk[32];
    for (int m = fvw; m < 32; m <<= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, m);
    if (threadIdx.x < 32) blk[threadIdx.x] = 0;
    __syncthreads();
    if (lane < fvw && bits) atomicOr(&blk[lane], bits);
    __syncthreads();
    if (warp == 0 && lane < fvw && fv_ok && blk[lane]) atomicOr(&unsat[fv], blk[lane]);
}

// --------------------------------------------------------- float check kernel
// Lane layout: lane = slot * fvw + lfv; the warp serves 32/fvw checks at a time
// (one per slot) over fvw frame vectors.  blockIdx.x walks check groups (so the
// resident blocks share one range of frames and their posterior gathers hit L2),
// blockIdx.y walks frame-vector ranges.
template <int ALGO, typename MsgT>
__global__ void __launch_bounds__(kCheckWarps * 32)
check_flood_f(DecArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw;
    const int slot = lane / fvw, lfv = lane - slot * fvw;
    const float *L = reinterpret_cast<const float *>(a.L);
    MsgT *msg = reinterpret_cast<MsgT *>(a.msg);
    unsigned long long units = 0;
    for (int64_t fb = blockIdx.y; fb * fvw < a.FV; fb += gridDim.y) {
        const int64_t fv = fb * fvw + lfv;
        const bool fv_ok = fv < a.FV;
        const uint32_t act = fv_ok ? active4(a.active, fv) : 0u;
        uint32_t unsat_bits = 0;
        if (act) {
            const int nact = __popc(act & 0x01010101u);
            const int64_t c0 = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
            for (int it = 0; it < kChecksPerWarp; ++it) {
                const int64_t c = c0 + it * slots + slot;
                if (c >= a.M) break;
                const int32_t beg = __ldg(a.rp + c), end = __ldg(a.rp + c + 1);
                const uint32_t sw = __ldg(a.sbits + c * a.W + ((4 * fv) >> 5));
                const uint32_t s4 = (sw >> ((4 * fv) & 31)) & 0xfu;
                uint32_t par = s4;          // syndrome xor hard decisions of L
                uint32_t neg = s4;          // syndrome xor signs of q
                float acc0[4], acc1[4];     // SP: sum of phi except the largest, largest phi
                int32_t arg[4];             //     OMS: min1, min2
                for (int i = 0; i < 4; ++i) {
                    acc0[i] = ALGO == kSP ? 0.0f : INFINITY;
                    acc1[i] = ALGO == kSP ? 0.0f : INFINITY;
                    arg[i] = -1;
                }
                for (int32_t e = beg; e < end; ++e) {
                    const int32_t v = __ldg(a.ci + e);
                    const F4 Lv = ld_f4(L + ((int64_t)v * a.FV + fv) * 4);
                    F4 mo = {{0.f, 0.f, 0.f, 0.f}};
                    if (a.do_msgs) mo = ld_msg(msg + ((int64_t)e * a.FV + fv) * 4);
                    for (int i = 0; i < 4; ++i) {
                        par ^= (uint32_t)(Lv.v[i] < 0.0f) << i;
                        const float q = Lv.v[i] - mo.v[i];
                        neg ^= (uint32_t)(q < 0.0f) << i;
                        if (ALGO == kSP) {
                            const float f = phi_f(fminf(fmaxf(fabsf(q), kAMin), kAMax));
                            if (f > acc1[i]) { acc0[i] += acc1[i]; acc1[i] = f; arg[i] = e; }
                            else acc0[i] += f;
                        } else {
                            const float m = fabsf(q);
                            if (m < acc0[i]) { acc1[i] = acc0[i]; acc0[i] = m; arg[i] = e; }
                            else if (m < acc1[i]) acc1[i] = m;
                        }
                    }
                }
                unsat_bits |= par;
                units += (unsigned long long)(end - beg) * nact;
                if (!a.do_msgs) continue;
                for (int32_t e = beg; e < end; ++e) {
                    const int32_t v = __ldg(a.ci + e);
                    const F4 Lv = ld_f4(L + ((int64_t)v * a.FV + fv) * 4);
                    MsgT *mp = msg + ((int64_t)e * a.FV + fv) * 4;
                    const F4 mo = ld_msg(mp);
                    F4 mn;
                    for (int i = 0; i < 4; ++i) {
                        const float q = Lv.v[i] - mo.v[i];
                        const bool sneg = ((neg >> i) & 1u) ^ (q < 0.0f);
                        float mag;
                        if (ALGO == kSP) {
                            const float f = phi_f(fminf(fmaxf(fabsf(q), kAMin), kAMax));
                            const float ex = (e == arg[i]) ? acc0[i] : acc0[i] + (acc1[i] - f);
                            mag = phi_f(fminf(fmaxf(ex, kAMin), kAMax));
                        } else {
                            mag = fmaxf(((e == arg[i]) ? acc1[i] : acc0[i]) - a.beta, 0.0f);
                        }
                        mn.v[i] = sneg ? -mag : mag;
                    }
                    st_msg(mp, mn);
                }
            }
            // only frames still decoding count
            uint32_t am = 0;
            for (int i = 0; i < 4; ++i) am |= (uint32_t)act_bit(act, i) << i;
            unsat_bits &= am;
        }
        if (a.early_stop || !a.do_msgs)
            publish_unsat(unsat_bits, fvw, lane, warp, fv, fv_ok, a.unsat_cur);
    }
    // messages read + written and the posterior gathered, per active edge-frame
    prof_add(a.prof, units, units * (a.do_msgs ? 2 * sizeof(MsgT) + 4 : 4));
}

// ----------------------------------------------------- integer check kernel
template <bool UNUSED>
__global__ void __launch_bounds__(kCheckWarps * 32)
check_flood_i(DecArgs a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw;
    const int slot = lane / fvw, lfv = lane - slot * fvw;
    const int16_t *L = reinterpret_cast<const int16_t *>(a.L);
    int8_t *msg = reinterpret_cast<int8_t *>(a.msg);
    unsigned long long units = 0;
    for (int64_t fb = blockIdx.y; fb * fvw < a.FV; fb += gridDim.y) {
        const int64_t fv = fb * fvw + lfv;
        const bool fv_ok = fv < a.FV;
        const uint32_t act = fv_ok ? active4(a.active, fv) : 0u;
        uint32_t unsat_bits = 0;
        if (act) {
            const int nact = __popc(act & 0x01010101u);
            const int64_t c0 = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
            for (int it = 0; it < kChecksPerWarp; ++it) {
                const int64_t c = c0 + it * slots + slot;
                if (c >= a.M) break;
                const int32_t beg = __ldg(a.rp + c), end = __ldg(a.rp + c + 1);
                const uint32_t sw = __ldg(a.sbits + c * a.W + ((4 * fv) >> 5));
                const uint32_t s4 = (sw >> ((4 * fv) & 31)) & 0xfu;
                uint32_t par = s4, neg = s4;
                int mn1[4], mn2[4], arg[4];
                for (int i = 0; i < 4; ++i) { mn1[i] = 1 << 20; mn2[i] = 1 << 20; arg[i] = -1; }
                for (int32_t e = beg; e < end; ++e) {
                    const int32_t v = __ldg(a.ci + e);
                    const I4 Lv = ld_i16x4(L + ((int64_t)v * a.FV + fv) * 4);
                    I4 mo = {{0, 0, 0, 0}};
                    if (a.do_msgs) mo = ld_i8x4(msg + ((int64_t)e * a.FV + fv) * 4);
                    for (int i = 0; i < 4; ++i) {
                        par ^= (uint32_t)(Lv.v[i] < 0) << i;
                        const int q = max(min(Lv.v[i] - mo.v[i], kQMax), -kQMax);
                        neg ^= (uint32_t)(q < 0) << i;
                        const int m = q < 0 ? -q : q;
                        if (m < mn1[i]) { mn2[i] = mn1[i]; mn1[i] = m; arg[i] = e; }
                        else if (m < mn2[i]) mn2[i] = m;
                    }
                }
                unsat_bits |= par;
                units += (unsigned long long)(end - beg) * nact;
                if (!a.do_msgs) continue;
                for (int32_t e = beg; e < end; ++e) {
                    const int32_t v = __ldg(a.ci + e);
                    const I4 Lv = ld_i16x4(L + ((int64_t)v * a.FV + fv) * 4);
                    int8_t *mp = msg + ((int64_t)e * a.FV + fv) * 4;
                    const I4 mo = ld_i8x4(mp);
                    I4 mn;
                    for (int i = 0; i < 4; ++i) {
                        const int q = max(min(Lv.v[i] - mo.v[i], kQMax), -kQMax);
                        const bool sneg = ((neg >> i) & 1u) ^ (q < 0);
                        const int mag = max(((e == arg[i]) ? mn2[i] : mn1[i]) - 1, 0);
                        mn.v[i] = sneg ? -mag : mag;
                    }
                    st_i8x4(mp, mn);
                }
            }
            uint32_t am = 0;
            for (int i = 0; i < 4; ++i) am |= (uint32_t)act_bit(act, i) << i;
            unsat_bits &= am;
        }
        if (a.early_stop || !a.do_msgs)
            publish_unsat(unsat_bits, fvw, lane, warp, fv, fv_ok, a.unsat_cur);
    }
    prof_add(a.prof, units, units * (a.do_msgs ? 4 : 2));
}

// ------------------------------------------------------------ variable kernels
// Retire frames whose stopping test passed on L^(t-1); update the rest:
// L_v = llr_v + sum of the messages on the edges of v (ascending edge order).
template <int PREC>
__global__ void __launch_bounds__(256) var_flood(DecArgs a) {
    const int64_t total = (int64_t)a.n * a.FV;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // per updated variable-frame: its messages, its channel LLR, the new posterior
    constexpr unsigned ms = PREC == kF32 ? 4 : (PREC == kF16 ? 2 : 1);
    constexpr unsigned cs = PREC == kI8 ? 1 : 4, ls = PREC == kI8 ? 2 : 4;
    unsigned long long units = 0, bytes = 0;
    for (int64_t item = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; item < total; item += stride) {
        const int64_t v = item / a.FV, fv = item - v * a.FV;
        const uint32_t act = active4(a.active, fv);
        if (!act) continue;
        uint32_t upd = 0;  // frames to update
        uint32_t done = 0; // frames retiring now
        const uint32_t u = a.early_stop ? __ldcg(a.unsat_cur + fv) : 0xfu;
        for (int i = 0; i < 4; ++i) {
            if (!act_bit(act, i)) continue;
            if (a.early_stop && !((u >> i) & 1u)) done |= 1u << i;
            else upd |= 1u << i;
        }
        if (v == 0) {
            for (int i = 0; i < 4; ++i)
                if ((done >> i) & 1u) {
                    a.active[4 * fv + i] = 0;
                    a.iters_i[4 * fv + i] = a.t - 1;
                }
            if (a.early_stop) a.unsat_next[fv] = 0;
        }
        if (!upd) continue;
        const int32_t vb = __ldg(a.vptr + v), ve = __ldg(a.vptr + v + 1);
        const unsigned nu = __popc(upd);
        units += nu;
        bytes += (unsigned long long)nu * ((ve - vb) * ms + cs + ls);
        if (PREC != kI8) {
            float *L = reinterpret_cast<float *>(a.L);
            const float *llr = reinterpret_cast<const float *>(a.llr_i);
            F4 s = ld_f4(llr + item * 4);
            for (int32_t k = vb; k < ve; ++k) {
                const int32_t e = __ldg(a.vedge + k);
                F4 m;
                if (PREC == kF32) m = ld_msg(reinterpret_cast<const float *>(a.msg) + ((int64_t)e * a.FV + fv) * 4);
                else m = ld_msg(reinterpret_cast<const __half *>(a.msg) + ((int64_t)e * a.FV + fv) * 4);
                for (int i = 0; i < 4; ++i) s.v[i] += m.v[i];
            }
            if (upd != 0xfu) {
                const F4 old = *reinterpret_cast<const F4 *>(L + item * 4);
                for (int i = 0; i < 4; ++i)
                    if (!((upd >> i) & 1u)) s.v[i] = old.v[i];
            }
            st_f4(L + item * 4, s);
        } else {
            int16_t *L = reinterpret_cast<int16_t *>(a.L);
            const I4 q = ld_i8x4(reinterpret_cast<const int8_t *>(a.llr_i) + item * 4);
            int s[4] = {q.v[0], q.v[1], q.v[2], q.v[3]};
            for (int32_t k = vb; k < ve; ++k) {
                const int32_t e = __ldg(a.vedge + k);
                const I4 m = ld_i8x4(reinterpret_cast<const int8_t *>(a.msg) + ((int64_t)e * a.FV + fv) * 4);
                for (int i = 0; i < 4; ++i) s[i] = max(min(s[i] + m.v[i], kPMax), -kPMax);
            }
            I4 r = {{s[0], s[1], s[2], s[3]}};
            if (upd != 0xfu) {
                const short4 o = *reinterpret_cast<const short4 *>(L + item * 4);
                const int ov[4] = {o.x, o.y, o.z, o.w};
                for (int i = 0; i < 4; ++i)
                    if (!((upd >> i) & 1u)) r.v[i] = ov[i];
            }
            st_i16x4(L + item * 4, r);
        }
    }
    prof_add(a.prof, units, bytes);
}

// ------------------------------------------------------- layout conversions
// llr [F][n] -> llr_i [n][Fp] and L [n][Fp]; padding frames get a
// confident all-zero word (they satisfy a zero syndrome at iteration 0).
template <int PREC>
__global__ void prep_llr(const float *__restrict__ llr, int32_t F, int32_t n, int64_t Fp, float step,
                         void *llr_i, void *L) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t v0 = (int64_t)blockIdx.x * 32, f0 = (int64_t)blockIdx.y * 32;
    for (int r = 0; r < 32; r += 8) {
        const int64_t f = f0 + ty + r, v = v0 + tx;
        float val = kLlrClip;
        if (f < F && v < n) val = llr[f * n + v];
        tile[ty + r][tx] = val;
    }
    __syncthreads();
    for (int r = 0; r < 32; r += 8) {
        const int64_t v = v0 + ty + r, f = f0 + tx;
        if (v >= n || f >= Fp) continue;
        const float val = tile[tx][ty + r];
        const int64_t o = v * Fp + f;
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
}

// synd [F][M] (bytes) -> sbits [M][W] (bit f%32 of word f/32).
__global__ void prep_synd(const uint8_t *__restrict__ synd, int32_t F, int32_t M, int64_t W,
                          uint32_t *__restrict__ sbits) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t w = blockIdx.y;
    const int64_t f = w * 32 + lane;
    const int64_t cbeg = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * 64;
    for (int64_t c = cbeg; c < cbeg + 64 && c < M; ++c) {
        const uint32_t bit = (f < F) ? (synd[f * M + c] & 1u) : 0u;
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == 0) sbits[c * W + w] = word;
    }
}

// per-frame state; `mask` marks the frames this decode owns (all real frames,
// or only the frames a low-precision pass left unsatisfied)
__global__ void init_state(int32_t F, int64_t Fp, const uint8_t *__restrict__ conv_prev,
                           uint8_t *active, uint8_t *mask, int32_t *iters_i, uint32_t *unsat0,
                           uint32_t *unsat1) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= Fp) return;
    const uint8_t a = (f < F) && (!conv_prev || !conv_prev[f]);
    active[f] = a;
    mask[f] = a;
    iters_i[f] = 0;
    if ((f & 3) == 0) {
        unsat0[f >> 2] = 0;
        unsat1[f >> 2] = 0;
    }
}

// `accumulate`: a re-decode adds its iterations to those of the first pass.
__global__ void finalize(int32_t F, int32_t T, int32_t accumulate, const uint8_t *__restrict__ mask,
                         const uint8_t *__restrict__ active, const int32_t *__restrict__ iters_i,
                         const uint32_t *__restrict__ unsat, int32_t *iters_out, uint8_t *conv_out) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= F || !mask[f]) return;
    const int32_t base = accumulate ? iters_out[f] : 0;
    if (active[f]) {
        iters_out[f] = base + T;
        conv_out[f] = !((unsat[f >> 2] >> (f & 3)) & 1u);
    } else {
        iters_out[f] = base + iters_i[f];
        conv_out[f] = 1;
    }
}

// L [n][Fp] -> bits [F][n] (+ posterior [F][n]) for the frames in `mask`.
template <int PREC>
__global__ void write_out(const void *Lp, int32_t F, int32_t n, int64_t Fp, float step,
                          const uint8_t *__restrict__ mask, uint8_t *bits, float *post) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t v0 = (int64_t)blockIdx.x * 32, f0 = (int64_t)blockIdx.y * 32;
    for (int r = 0; r < 32; r += 8) {
        const int64_t v = v0 + ty + r, f = f0 + tx;
        float val = 0.0f;
        if (v < n && f < Fp) {
            if (PREC == kI8) val = (float)reinterpret_cast<const int16_t *>(Lp)[v * Fp + f];
            else val = reinterpret_cast<const float *>(Lp)[v * Fp + f];
        }
        tile[tx][ty + r] = val;
    }
    __syncthreads();
    for (int r = 0; r < 32; r += 8) {
        const int64_t f = f0 + ty + r, v = v0 + tx;
        if (f >= F || v >= n || !mask[f]) continue;
        const float val = tile[ty + r][tx];
        bits[f * n + v] = val < 0.0f ? 1 : 0;
        if (post) post[f * n + v] = PREC == kI8 ? val * step : val;
    }
}

// ------------------------------------------------------------------ layout
struct Layout {
    int64_t Fp, FV, W;
    size_t llr_i, L, msg, sbits, active, mask, unsat0, unsat1, iters, total;
};

static Layout make_layout(const CodeDev &d, int32_t F, int prec) {
    Layout l;
    l.Fp = align_up((size_t)(F > 0 ? F : 1), 4);
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
    l.unsat0 = take((size_t)l.FV * 4);
    l.unsat1 = take((size_t)l.FV * 4);
    l.iters = take((size_t)l.Fp * 4);
    l.total = off;
    return l;
}

static bool opts_ok(const qkdrec_decode_opts *o) {
    return o && o->algo >= 0 && o->algo <= 2 && o->prec >= 0 && o->prec <= 2 && o->max_iter >= 0 &&
           isfinite(o->offset) && o->offset >= 0.0f && isfinite(o->llr_step) && o->llr_step > 0.0f;
}

static size_t workspace_for(const CodeDev &d, int32_t F, const qkdrec_decode_opts *o) {
    size_t b = make_layout(d, F, o->prec).total;
    if (o->fallback_f32 && o->prec != kF32) {
        size_t b32 = make_layout(d, F, kF32).total;
        if (b32 > b) b = b32;
    }
    return b;
}

struct Prepared {
    uint32_t *unsat[2];
    uint8_t *mask;
};

// Shared set-up of one decode pass: per-frame state, interleaved LLRs and
// posteriors, packed syndromes, zero messages, and the launch geometry.
static qkdrec_status prepare(const CodeDev &d, const float *llr, const uint8_t *synd, int32_t F,
                             const qkdrec_decode_opts &o, int prec, const uint8_t *conv_prev, char *ws,
                             const Layout &l, cudaStream_t st, DecArgs &a, Prepared &pr) {
    a.rp = d.rp;
    a.ci = d.ci;
    a.vptr = d.vptr;
    a.vedge = d.vedge;
    a.sbits = reinterpret_cast<const uint32_t *>(ws + l.sbits);
    a.active = reinterpret_cast<uint8_t *>(ws + l.active);
    a.iters_i = reinterpret_cast<int32_t *>(ws + l.iters);
    a.L = ws + l.L;
    a.msg = ws + l.msg;
    a.llr_i = ws + l.llr_i;
    a.FV = l.FV;
    a.W = l.W;
    a.n = d.n;
    a.M = d.M;
    a.fvw = 1;
    while (a.fvw < 32 && a.fvw < l.FV) a.fvw <<= 1;
    a.t = 0;
    a.do_msgs = 1;
    a.early_stop = o.early_stop ? 1 : 0;
    a.beta = o.offset;
    a.prof = nullptr;
    pr.unsat[0] = reinterpret_cast<uint32_t *>(ws + l.unsat0);
    pr.unsat[1] = reinterpret_cast<uint32_t *>(ws + l.unsat1);
    pr.mask = reinterpret_cast<uint8_t *>(ws + l.mask);
    a.unsat_cur = pr.unsat[0];
    a.unsat_next = pr.unsat[1];

    {
        prof::Scope ps(prof::kPrep, st);
        init_state<<<(unsigned)ceil_div(l.Fp, 256), 256, 0, st>>>(F, l.Fp, conv_prev, a.active, pr.mask,
                                                                 a.iters_i, pr.unsat[0], pr.unsat[1]);
    }
    QKD_LAUNCHED("init_state");
    {
        prof::Scope ps(prof::kPrep, st);
        dim3 blk(32, 8), grd((unsigned)ceil_div(d.n, 32), (unsigned)ceil_div(l.Fp, 32));
        if (prec == kI8) prep_llr<kI8><<<grd, blk, 0, st>>>(llr, F, d.n, l.Fp, o.llr_step, ws + l.llr_i, ws + l.L);
        else prep_llr<kF32><<<grd, blk, 0, st>>>(llr, F, d.n, l.Fp, o.llr_step, ws + l.llr_i, ws + l.L);
        QKD_LAUNCHED("prep_llr");
    }
    {
        prof::Scope ps(prof::kPrep, st);
        dim3 grd((unsigned)ceil_div(d.M, 8 * 64), (unsigned)l.W);
        prep_synd<<<grd, 256, 0, st>>>(synd, F, d.M, l.W, reinterpret_cast<uint32_t *>(ws + l.sbits));
        QKD_LAUNCHED("prep_synd");
    }
    const size_t ms = prec == kF32 ? 4 : (prec == kF16 ? 2 : 1);
    QKD_CUDA(cudaMemsetAsync(ws + l.msg, 0, (size_t)d.E * l.Fp * ms, st));
    return QKDREC_OK;
}

// Shared tail: iteration counts / converged flags, then bits and posteriors
// back to the frame-major output layout.
static qkdrec_status finish(const CodeDev &d, int32_t F, int T, int prec, const qkdrec_decode_opts &o,
                            const uint8_t *conv_prev, char *ws, const Layout &l, const Prepared &pr,
                            const DecArgs &a, int final_buf, uint8_t *bits_out, int32_t *iters_out,
                            uint8_t *conv_out, float *post_out, cudaStream_t st) {
    {
        prof::Scope ps(prof::kFinish, st);
        finalize<<<(unsigned)ceil_div(F, 256), 256, 0, st>>>(F, T, conv_prev ? 1 : 0, pr.mask, a.active,
                                                             a.iters_i, pr.unsat[final_buf], iters_out, conv_out);
    }
    QKD_LAUNCHED("finalize");
    prof::Scope ps(prof::kFinish, st);
    dim3 blk(32, 8), grd((unsigned)ceil_div(d.n, 32), (unsigned)ceil_div(l.Fp, 32));
    if (prec == kI8) write_out<kI8><<<grd, blk, 0, st>>>(ws + l.L, F, d.n, l.Fp, o.llr_step, pr.mask, bits_out, post_out);
    else write_out<kF32><<<grd, blk, 0, st>>>(ws + l.L, F, d.n, l.Fp, o.llr_step, pr.mask, bits_out, post_out);
    QKD_LAUNCHED("write_out");
    return QKDREC_OK;
}

// One flooding decode pass over the frames selected by conv_prev (NULL = all).
static qkdrec_status run_flood(const CodeDev &d, const float *llr, const uint8_t *synd, int32_t F,
                               const qkdrec_decode_opts &o, int prec, const uint8_t *conv_prev,
                               uint8_t *bits_out, int32_t *iters_out, uint8_t *conv_out,
                               float *post_out, char *ws, cudaStream_t st) {
    const Layout l = make_layout(d, F, prec);
    DecArgs a;
    Prepared pr;
    qkdrec_status s = prepare(d, llr, synd, F, o, prec, conv_prev, ws, l, st, a, pr);
    if (s != QKDREC_OK) return s;
    const int slots = 32 / a.fvw;
    const int64_t checks_per_block = (int64_t)kCheckWarps * kChecksPerWarp * slots;
    const int64_t fblocks = ceil_div(l.FV, a.fvw);
    dim3 cgrid((unsigned)ceil_div(d.M, checks_per_block), (unsigned)(fblocks < 65535 ? fblocks : 65535));
    const int64_t vitems = (int64_t)d.n * l.FV;
    const unsigned vgrid = (unsigned)std::min<int64_t>(ceil_div(vitems, 256), (int64_t)sm_count() * 64);

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
        if (prec == kI8) check_flood_i<true><<<cgrid, kCheckWarps * 32, 0, st>>>(a);
        else if (o.algo == QKDREC_SP_FLOOD) {
            if (prec == kF32) check_flood_f<kSP, float><<<cgrid, kCheckWarps * 32, 0, st>>>(a);
            else check_flood_f<kSP, __half><<<cgrid, kCheckWarps * 32, 0, st>>>(a);
        } else {
            if (prec == kF32) check_flood_f<kOMS, float><<<cgrid, kCheckWarps * 32, 0, st>>>(a);
            else check_flood_f<kOMS, __half><<<cgrid, kCheckWarps * 32, 0, st>>>(a);
        }
    };
    for (int t = 1; t <= o.max_iter; ++t) {
        check(t, 1);
        QKD_LAUNCHED("check_flood");
        a.t = t;
        {
            const int kind = prec == kI8 ? prof::kVarI8 : (prec == kF16 ? prof::kVarF16 : prof::kVarF32);
            a.prof = prof::counters(kind);
            prof::Scope ps(kind, st);
            if (prec == kI8) var_flood<kI8><<<vgrid, 256, 0, st>>>(a);
            else if (prec == kF16) var_flood<kF16><<<vgrid, 256, 0, st>>>(a);
            else var_flood<kF32><<<vgrid, 256, 0, st>>>(a);
        }
        QKD_LAUNCHED("var_flood");
    }
    // stopping test on the final posteriors (parity buffer (T+1)&1 is clear)
    const int T = o.max_iter;
    a.early_stop = 1;
    check(T + 1, 0);
    QKD_LAUNCHED("check_flood(parity)");
    return finish(d, F, T, prec, o, conv_prev, ws, l, pr, a, (T + 1) & 1, bits_out, iters_out, conv_out,
                  post_out, st);
}

#include "decode_layered.cuh"

}  // namespace qkd

using namespace qkd;

extern "C" {

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
    clear_error();
    if (!code) QKD_FAIL(QKDREC_ERR_ARG, "code is NULL");
    if (F < 0) QKD_FAIL(QKDREC_ERR_ARG, "F < 0");
    if (!opts_ok(opts)) QKD_FAIL(QKDREC_ERR_ARG, "bad decode options");
    const qkdrec_decode_opts o = *opts;
    if (o.prec == QKDREC_I8SAT && o.algo == QKDREC_SP_FLOOD)
        QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "integer messages need an offset min-sum algorithm");
    if (F == 0) return QKDREC_OK;
    if (F > kMaxFrames) QKD_FAIL(QKDREC_ERR_ARG, "F=%d above the %d frames of one launch", F, kMaxFrames);
    if (!llr || !synd || !bits_out || !iters_out || !conv_out) QKD_FAIL(QKDREC_ERR_ARG, "NULL input/output");
    if (!workspace) QKD_FAIL(QKDREC_ERR_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) % 256) QKD_FAIL(QKDREC_ERR_ARG, "workspace not 256-byte aligned");
    const size_t need = workspace_for(code->d, F, &o);
    if (workspace_bytes < need) QKD_FAIL(QKDREC_ERR_ARG, "workspace %zu bytes < %zu needed", workspace_bytes, need);
    const CodeDev &d = code->d;
    cudaStream_t st = as_stream(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    qkdrec_status s;
    auto pass = [&](int prec, const uint8_t *conv_prev) {
        if (o.algo == QKDREC_OMS_LAYERED)
            return run_layered(d, llr, synd, F, o, prec, conv_prev, bits_out, iters_out, conv_out, post_out, ws, st);
        return run_flood(d, llr, synd, F, o, prec, conv_prev, bits_out, iters_out, conv_out, post_out, ws, st);
    };
    if ((s = pass(o.prec, nullptr)) != QKDREC_OK) return s;
    // FP32 re-decode of the frames a low-precision pass left unsatisfied
    if (o.fallback_f32 && o.prec != QKDREC_F32) {
        if ((s = pass(QKDREC_F32, conv_out)) != QKDREC_OK) return s;
    }
    return QKDREC_OK;
}

}  // extern "C"

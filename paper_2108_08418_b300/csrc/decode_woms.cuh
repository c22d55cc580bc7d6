// Unrolled weighted offset min-sum and its adjoint (included at the end of decode.cu).
//
// Forward, T flooding iterations without a stopping test; iteration t uses the
// weights of its check's degree class (class 0 = the code's smallest check
// degree):
//   q_e = L^{t-1}_{v(e)} - m^{t-1}_e,
//   m^t_e = (-1)^{s_c} prod_{other edges} sgn(q) * alpha[t][cls] * max(mn_e - beta[t][cls], 0),
//   mn_e = min over the other edges of |q|,   L^t_v = llr_v + sum_{e at v} m^t_e.
// Loss = mean over frames and variables of b softplus(L^T) + (1 - b) softplus(-L^T),
// the binary cross-entropy of P(b = 1) = sigmoid(-L^T) against the target bits.
//
// Adjoint: the gradient of m^t_e flows (i) through alpha and beta of the
// iteration and (ii) to |q| of the edge that holds the minimum over the other
// edges (ties: the lowest edge index; max(x, 0)' = 0 at x <= 0; signs carry no
// gradient).  Per iteration, going backwards:
//   g_e   = gm_e + gL^t_{v(e)}       (gm_e: gradient of m^t_e through q^{t+1})
//   check backward: galpha, gbeta, and gq_e (non-zero on the two argmin edges)
//   variable backward: gL^{t-1}_v = sum_{e at v} gq_e,  gm_e = -gq_e.
// Checkpointing: the forward keeps m^t at t = K, 2K, ... < T; the backward
// recomputes each K-iteration segment from its checkpoint, newest first.
//
// Layout: the decoder's frame-block-major arrays with 32-frame blocks, one
// frame per lane.

namespace qkd {

constexpr int kWomsLg = 5;  // 32-frame blocks

struct WomsArgs {
    const int32_t *rp, *ci, *vptr, *vedge;
    const uint32_t *sbits;
    const float *alpha, *beta;   // DEVICE [T][2]
    const float *llr_i;          // [n][Fp]
    const uint8_t *tgt_i;        // [n][Fp] target bits
    int64_t Fp, W, E;
    int32_t n, M, F, dmin, t, fvw;
    const float *L_in;           // L^{t-1}
    const float *m_in;           // m^{t-1}
    float *m_out;                // m^t (forward)
    float *L_out;                // L^t (forward variable kernel)
    float *gL;                   // gradient w.r.t. L^t (in), L^{t-1} (out of the variable kernel)
    float *gm;                   // gradient w.r.t. m^t through q^{t+1}; overwritten with -gq^t
    double *grads;               // [T][2 classes][2] (alpha, beta)
    double *loss;
    unsigned long long *prof;
};

// Column of a check's edges and the frame of this lane.
struct WomsLane {
    int lane, warp, slot, lfv, slots;
};

// q of every edge of check c for frame f0 (stashed in shared memory), the sign
// parity, and the two smallest |q| with their lowest-index positions.
struct CheckState {
    int32_t beg, d, am1, am2;
    float mn1, mn2;
    uint32_t neg, sg;
};

__device__ __forceinline__ CheckState woms_scan(const WomsArgs &a, int64_t c, int64_t f0, int64_t bL,
                                                int64_t bM, float *my) {
    CheckState st;
    st.beg = __ldg(a.rp + c);
    st.d = __ldg(a.rp + c + 1) - st.beg;
    st.neg = (__ldg(a.sbits + c * a.W + (f0 >> 5)) >> (f0 & 31)) & 1u;
    st.sg = 0;
    st.mn1 = INFINITY;
    st.mn2 = INFINITY;
    st.am1 = -1;
    st.am2 = -1;
    constexpr int CH = 8;
    for (int k0 = 0; k0 < st.d; k0 += CH) {
        float Lv[CH], mo[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int32_t e = st.beg + min(k0 + j, st.d - 1);
            Lv[j] = __ldg(a.L_in + bL + ((uint32_t)__ldg(a.ci + e) << kWomsLg));
            mo[j] = a.m_in ? __ldcs(a.m_in + bM + ((uint32_t)e << kWomsLg)) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int k = k0 + j;
            if (k >= st.d) break;
            const float q = Lv[j] - mo[j];
            my[k * 32] = q;
            const uint32_t sb = q < 0.0f;
            st.sg |= sb << k;
            st.neg ^= sb;
            const float m = fabsf(q);
            if (m < st.mn1) { st.mn2 = st.mn1; st.am2 = st.am1; st.mn1 = m; st.am1 = k; }
            else if (m < st.mn2) { st.mn2 = m; st.am2 = k; }
        }
    }
    return st;
}

__global__ void __launch_bounds__(kCheckWarps * 32)
woms_check_fwd(WomsArgs a) {
    extern __shared__ float qst[];  // [kCheckWarps][kStash][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw, slot = lane / fvw, lfv = lane - slot * fvw;
    float *my = qst + (warp * kStash) * 32 + lane;
    unsigned long long units = 0;
    for (int64_t fb = blockIdx.y; fb * fvw < a.Fp; fb += gridDim.y) {
        const int64_t f0 = fb * fvw + lfv;
        if (f0 >= a.Fp) continue;
        const int64_t bL = fpos(0, a.n, f0, kWomsLg), bM = fpos(0, a.E, f0, kWomsLg);
        const int64_t c0 = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
        for (int it = 0; it < kChecksPerWarp; ++it) {
            const int64_t c = c0 + it * slots + slot;
            if (c >= a.M) break;
            const CheckState st = woms_scan(a, c, f0, bL, bM, my);
            const int cls = st.d == a.dmin ? 0 : 1;
            const float al = __ldg(a.alpha + 2 * (a.t - 1) + cls), be = __ldg(a.beta + 2 * (a.t - 1) + cls);
            units += st.d;
            for (int k = 0; k < st.d; ++k) {
                const float mn = k == st.am1 ? st.mn2 : st.mn1;
                const float mag = al * fmaxf(mn - be, 0.0f);
                const bool sneg = (st.neg ^ (st.sg >> k)) & 1u;
                __stcs(a.m_out + bM + ((uint32_t)(st.beg + k) << kWomsLg), sneg ? -mag : mag);
            }
        }
    }
    prof_add(a.prof, units, units * 12);
}

// L^t = llr + sum of m^t over the variable's edges (all frames, no stopping test).
__global__ void __launch_bounds__(256) woms_var_fwd(WomsArgs a) {
    const int64_t total = (int64_t)a.n * a.Fp;
    unsigned long long units = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / a.Fp, f = i - v * a.Fp;
        const int64_t pv = fpos(v, a.n, f, kWomsLg), bM = fpos(0, a.E, f, kWomsLg);
        float s = __ldg(a.llr_i + pv);
        for (int32_t k = __ldg(a.vptr + v), ke = __ldg(a.vptr + v + 1); k < ke; ++k)
            s += __ldcs(a.m_out + bM + ((uint32_t)__ldg(a.vedge + k) << kWomsLg));
        a.L_out[pv] = s;
        ++units;
    }
    prof_add(a.prof, units, units * 20);
}

// Loss of L^T and its gradient gL = (b sigmoid(L) - (1 - b) sigmoid(-L)) / (F n).
__global__ void __launch_bounds__(256) woms_loss(WomsArgs a, int want_grad) {
    __shared__ double part[8];
    const int64_t total = (int64_t)a.n * a.Fp;
    const double scale = 1.0 / ((double)a.F * (double)a.n);
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / a.Fp, f = i - v * a.Fp;
        const int64_t pv = fpos(v, a.n, f, kWomsLg);
        if (f >= a.F) {
            if (want_grad) a.gL[pv] = 0.0f;
            continue;
        }
        const float L = a.L_in[pv];
        const bool b = a.tgt_i[pv] & 1;
        // softplus(x) = max(x, 0) + log1p(exp(-|x|)); sigmoid(x) = 1 / (1 + exp(-x))
        const float x = b ? L : -L;
        acc += (double)(fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x))));
        if (want_grad) {
            const float sg = 1.0f / (1.0f + expf(-x));      // sigmoid(x)
            a.gL[pv] = (float)scale * (b ? sg : -sg);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        atomicAdd(a.loss, s * scale);
    }
}

// Check backward of iteration t: per edge g = gm + gL^t[v]; accumulates the
// alpha/beta gradients of the iteration and writes gm_e = -gq_e.
__global__ void __launch_bounds__(kCheckWarps * 32)
woms_check_bwd(WomsArgs a) {
    extern __shared__ float qst[];  // [kCheckWarps][kStash][32]
    __shared__ double red[kCheckWarps][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw, slot = lane / fvw, lfv = lane - slot * fvw;
    float *my = qst + (warp * kStash) * 32 + lane;
    float ga[2] = {0.f, 0.f}, gb[2] = {0.f, 0.f};
    unsigned long long units = 0;
    for (int64_t fb = blockIdx.y; fb * fvw < a.Fp; fb += gridDim.y) {
        const int64_t f0 = fb * fvw + lfv;
        if (f0 >= a.Fp) continue;
        const int64_t bL = fpos(0, a.n, f0, kWomsLg), bM = fpos(0, a.E, f0, kWomsLg);
        const int64_t c0 = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
        for (int it = 0; it < kChecksPerWarp; ++it) {
            const int64_t c = c0 + it * slots + slot;
            if (c >= a.M) break;
            const CheckState st = woms_scan(a, c, f0, bL, bM, my);
            const int cls = st.d == a.dmin ? 0 : 1;
            const float al = __ldg(a.alpha + 2 * (a.t - 1) + cls), be = __ldg(a.beta + 2 * (a.t - 1) + cls);
            const float s1 = my[st.am1 * 32] < 0.0f ? -1.0f : 1.0f;   // sgn(q) of the two argmin edges
            const float s2 = my[st.am2 * 32] < 0.0f ? -1.0f : 1.0f;
            float g1 = 0.0f, g2 = 0.0f;                              // gradient of |q| at am1, am2
            units += st.d;
            for (int k = 0; k < st.d; ++k) {
                const int32_t e = st.beg + k;
                const float g = a.gm[bM + ((uint32_t)e << kWomsLg)] +
                                a.gL[bL + ((uint32_t)__ldg(a.ci + e) << kWomsLg)];
                const float sigma = ((st.neg ^ (st.sg >> k)) & 1u) ? -1.0f : 1.0f;
                const bool first = k == st.am1;
                const float x = (first ? st.mn2 : st.mn1) - be;
                const float relu = fmaxf(x, 0.0f);
                ga[cls] += g * sigma * relu;
                if (x > 0.0f) {
                    const float gr = g * sigma * al;
                    gb[cls] -= gr;
                    if (first) g2 += gr;   // the minimum over the others is at am2
                    else g1 += gr;
                }
            }
            for (int k = 0; k < st.d; ++k) {
                const float gq = k == st.am1 ? g1 * s1 : (k == st.am2 ? g2 * s2 : 0.0f);
                a.gm[bM + ((uint32_t)(st.beg + k) << kWomsLg)] = -gq;
            }
        }
    }
    // block reduction of the four gradient sums, then one FP64 atomic each
    float v4[4] = {ga[0], gb[0], ga[1], gb[1]};
    for (int i = 0; i < 4; ++i)
        for (int o = 16; o > 0; o >>= 1) v4[i] += __shfl_xor_sync(0xffffffffu, v4[i], o);
    if (lane == 0)
        for (int i = 0; i < 4; ++i) red[warp][i] = (double)v4[i];
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kCheckWarps; ++w) s += red[w][threadIdx.x];
        // grads layout [t][cls][alpha/beta]
        const int cls = threadIdx.x >> 1, ab = threadIdx.x & 1;
        if (s != 0.0) atomicAdd(a.grads + 4 * (a.t - 1) + 2 * cls + ab, s);
    }
    prof_add(a.prof, units, units * 20);
}

// Variable backward: gL^{t-1}_v = sum_{e at v} gq_e = -sum gm_e.
__global__ void __launch_bounds__(256) woms_var_bwd(WomsArgs a) {
    const int64_t total = (int64_t)a.n * a.Fp;
    unsigned long long units = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / a.Fp, f = i - v * a.Fp;
        const int64_t pv = fpos(v, a.n, f, kWomsLg), bM = fpos(0, a.E, f, kWomsLg);
        float s = 0.0f;
        for (int32_t k = __ldg(a.vptr + v), ke = __ldg(a.vptr + v + 1); k < ke; ++k)
            s -= a.gm[bM + ((uint32_t)__ldg(a.vedge + k) << kWomsLg)];
        a.gL[pv] = s;
        ++units;
    }
    prof_add(a.prof, units, units * 16);
}

__global__ void prep_target(const uint8_t *__restrict__ tgt, int32_t F, int32_t n, int64_t Fp, uint8_t *out) {
    const int64_t total = (int64_t)n * Fp;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / Fp, f = i - v * Fp;
        out[fpos(v, n, f, kWomsLg)] = f < F ? (tgt[f * n + v] & 1) : 0;
    }
}

__global__ void grads_out(const double *g, int32_t T, float *galpha, float *gbeta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * T) return;
    const int t = i >> 1, cls = i & 1;
    galpha[i] = (float)g[4 * t + 2 * cls + 0];
    gbeta[i] = (float)g[4 * t + 2 * cls + 1];
}

__global__ void copy_loss(const double *l, float *out) { *out = (float)*l; }

// L [n][Fp] (32-frame blocks) -> post [F][n]
__global__ void write_post(const float *__restrict__ L, int32_t F, int32_t n, int64_t Fp, int lg, float *post) {
    __shared__ float tile[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t v0 = (int64_t)blockIdx.x * 32, f0 = (int64_t)blockIdx.y * 32;
    for (int r = 0; r < 32; r += 8) {
        const int64_t v = v0 + ty + r, f = f0 + tx;
        tile[tx][ty + r] = (v < n && f < Fp) ? L[fpos(v, n, f, lg)] : 0.0f;
    }
    __syncthreads();
    for (int r = 0; r < 32; r += 8) {
        const int64_t f = f0 + ty + r, v = v0 + tx;
        if (f < F && v < n) post[f * n + v] = tile[ty + r][tx];
    }
}

// --------------------------------------------------------------- host side
struct WomsLayout {
    int64_t Fp, W;
    int nseg, nck;
    size_t llr_i, tgt_i, sbits, ckpt, seg_m, seg_L, gL, gm, grads, loss, total;
};

static WomsLayout woms_layout(const CodeDev &d, int32_t F, int32_t T, int32_t K) {
    WomsLayout l;
    l.Fp = align_up((size_t)(F > 0 ? F : 1), 32);
    l.W = l.Fp / 32;
    l.nseg = (int)ceil_div(T, K);
    l.nck = l.nseg > 0 ? l.nseg - 1 : 0;
    const size_t me = (size_t)d.E * l.Fp * 4, ve = (size_t)d.n * l.Fp * 4;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    l.llr_i = take(ve);
    l.tgt_i = take((size_t)d.n * l.Fp);
    l.sbits = take((size_t)d.M * l.W * 4);
    l.ckpt = take(me * (size_t)l.nck);
    l.seg_m = take(me * (size_t)(K + 1));
    l.seg_L = take(ve * (size_t)(K + 1));
    l.gL = take(ve);
    l.gm = take(me);
    l.grads = take(sizeof(double) * 4 * (size_t)(T > 0 ? T : 1));
    l.loss = take(sizeof(double));
    l.total = off;
    return l;
}

static WomsArgs woms_args(const CodeDev &d, int32_t F, const float *alpha, const float *beta, char *ws,
                          const WomsLayout &l) {
    WomsArgs a;
    a.rp = d.rp;
    a.ci = d.ci;
    a.vptr = d.vptr;
    a.vedge = d.vedge;
    a.sbits = reinterpret_cast<const uint32_t *>(ws + l.sbits);
    a.alpha = alpha;
    a.beta = beta;
    a.llr_i = reinterpret_cast<const float *>(ws + l.llr_i);
    a.tgt_i = reinterpret_cast<const uint8_t *>(ws + l.tgt_i);
    a.Fp = l.Fp;
    a.W = l.W;
    a.E = d.E;
    a.n = d.n;
    a.M = d.M;
    a.F = F;
    a.dmin = d.dc_min;
    a.t = 0;
    a.L_in = a.m_in = nullptr;
    a.m_out = a.L_out = a.gL = a.gm = nullptr;
    a.grads = reinterpret_cast<double *>(ws + l.grads);
    a.loss = reinterpret_cast<double *>(ws + l.loss);
    a.prof = nullptr;
    Geom g = check_geom(l.Fp, 1, d.M);
    a.fvw = g.fvw;
    return a;
}

static qkdrec_status woms_check(const CodeDev &d, int32_t F, int32_t T, int32_t K, const void *ws) {
    if (T < 1 || T > 1000) QKD_FAIL(QKDREC_ERR_ARG, "iterations T=%d outside [1, 1000]", T);
    if (K < 1) QKD_FAIL(QKDREC_ERR_ARG, "checkpoint interval %d < 1", K);
    if (F < 1 || F > kMaxFrames) QKD_FAIL(QKDREC_ERR_ARG, "F=%d outside [1, %d]", F, kMaxFrames);
    if (d.dc_max > kStash) QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "check degree %d above %d", d.dc_max, kStash);
    if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) QKD_FAIL(QKDREC_ERR_ARG, "workspace NULL or not 256-byte aligned");
    return QKDREC_OK;
}

// Forward iterations t0+1 .. t1 from (L^{t0} in Lbuf[0], m^{t0} in mbuf[0]); with
// ring = true the results go to Lbuf[t - t0], mbuf[t - t0], otherwise they
// alternate between buffers 0 and 1 (plain forward).
static void woms_forward_range(WomsArgs a, const CodeDev &d, const WomsLayout &l, char *ws, int t0, int t1,
                               bool ring, int K, cudaStream_t st) {
    const size_t me = (size_t)d.E * l.Fp, ve = (size_t)d.n * l.Fp;
    float *mb = reinterpret_cast<float *>(ws + l.seg_m), *Lb = reinterpret_cast<float *>(ws + l.seg_L);
    const Geom g = check_geom(l.Fp, 1, d.M);
    const size_t stash = (size_t)kCheckWarps * kStash * 32 * sizeof(float);
    const unsigned vgrid = (unsigned)std::min<int64_t>(ceil_div((int64_t)d.n * l.Fp, 256), (int64_t)sm_count() * 32);
    for (int t = t0 + 1; t <= t1; ++t) {
        const int i_in = ring ? t - 1 - t0 : (t - 1 - t0) & 1, i_out = ring ? t - t0 : (t - t0) & 1;
        a.t = t;
        a.L_in = Lb + ve * i_in;
        a.m_in = (t == 1) ? nullptr : mb + me * i_in;
        a.m_out = mb + me * i_out;
        a.L_out = Lb + ve * i_out;
        a.prof = prof::counters(prof::kWomsFwd);
        {
            prof::Scope ps(prof::kWomsFwd, st);
            woms_check_fwd<<<g.grid, kCheckWarps * 32, stash, st>>>(a);
        }
        a.prof = prof::counters(prof::kWomsVar);
        {
            prof::Scope ps(prof::kWomsVar, st);
            woms_var_fwd<<<vgrid, 256, 0, st>>>(a);
        }
        // keep the checkpoints m^{K}, m^{2K}, ... below T
        if (!ring && t % K == 0 && t / K <= l.nck)
            cudaMemcpyAsync(ws + l.ckpt + (size_t)(t / K - 1) * me * 4, a.m_out, me * 4, cudaMemcpyDeviceToDevice, st);
    }
}

static qkdrec_status woms_prepare(const CodeDev &d, const float *llr, const uint8_t *synd, const uint8_t *target,
                                  int32_t F, char *ws, const WomsLayout &l, cudaStream_t st) {
    prof::Scope ps(prof::kPrep, st);
    dim3 blk(32, 8), grd((unsigned)ceil_div(d.n, 32), (unsigned)std::min<int64_t>(ceil_div(l.Fp, 32), 65535));
    prep_llr<kF32><<<grd, blk, 0, st>>>(llr, F, d.n, l.Fp, kWomsLg, 1.0f, ws + l.llr_i, ws + l.seg_L);
    prep_target<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)d.n * l.Fp, 256), 65535), 256, 0, st>>>(
        target, F, d.n, l.Fp, reinterpret_cast<uint8_t *>(ws + l.tgt_i));
    dim3 sg((unsigned)ceil_div(d.M, 8 * 64), (unsigned)std::min<int64_t>(l.W, 65535));
    prep_synd<<<sg, 256, 0, st>>>(synd, F, d.M, l.W, reinterpret_cast<uint32_t *>(ws + l.sbits));
    QKD_LAUNCHED("woms prepare");
    return QKDREC_OK;
}

}  // namespace qkd

extern "C" {

qkdrec_status qkdrec_woms_workspace_size(qkdrec_code_t code, int32_t F, int32_t T, int32_t ckpt_every,
                                         size_t *bytes) {
    clear_error();
    if (!code || !bytes) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    if (F < 1 || T < 1 || ckpt_every < 1) QKD_FAIL(QKDREC_ERR_ARG, "F, T and ckpt_every must be >= 1");
    *bytes = woms_layout(code->d, F, T, ckpt_every).total;
    return QKDREC_OK;
}

qkdrec_status qkdrec_woms_forward(qkdrec_code_t code, const float *llr, const uint8_t *synd, const uint8_t *target,
                                  int32_t F, int32_t T, const float *alpha, const float *beta, int32_t ckpt_every,
                                  float *loss_out, float *post_out, void *workspace, size_t workspace_bytes,
                                  void *stream) {
    clear_error();
    if (!code || !llr || !synd || !target || !alpha || !beta || !loss_out) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    const CodeDev &d = code->d;
    qkdrec_status s = woms_check(d, F, T, ckpt_every, workspace);
    if (s != QKDREC_OK) return s;
    const WomsLayout l = woms_layout(d, F, T, ckpt_every);
    if (workspace_bytes < l.total) QKD_FAIL(QKDREC_ERR_ARG, "workspace %zu < %zu bytes", workspace_bytes, l.total);
    cudaStream_t st = as_stream(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    if ((s = woms_prepare(d, llr, synd, target, F, ws, l, st)) != QKDREC_OK) return s;
    WomsArgs a = woms_args(d, F, alpha, beta, ws, l);
    woms_forward_range(a, d, l, ws, 0, T, false, ckpt_every, st);
    QKD_LAUNCHED("woms forward");
    // final posteriors are in seg_L[T & 1]
    const float *LT = reinterpret_cast<const float *>(ws + l.seg_L) + (size_t)d.n * l.Fp * (T & 1);
    QKD_CUDA(cudaMemsetAsync(ws + l.loss, 0, sizeof(double), st));
    a.L_in = LT;
    {
        prof::Scope ps(prof::kFinish, st);
        woms_loss<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)d.n * l.Fp, 256), 4096), 256, 0, st>>>(a, 0);
        copy_loss<<<1, 1, 0, st>>>(a.loss, loss_out);
        if (post_out) {
            dim3 blk(32, 8), grd((unsigned)ceil_div(d.n, 32), (unsigned)std::min<int64_t>(ceil_div(l.Fp, 32), 65535));
            write_post<<<grd, blk, 0, st>>>(LT, F, d.n, l.Fp, kWomsLg, post_out);
        }
    }
    QKD_LAUNCHED("woms loss");
    return QKDREC_OK;
}

qkdrec_status qkdrec_woms_backward(qkdrec_code_t code, const float *llr, const uint8_t *synd, const uint8_t *target,
                                   int32_t F, int32_t T, const float *alpha, const float *beta, int32_t ckpt_every,
                                   float *grad_alpha, float *grad_beta, void *workspace, size_t workspace_bytes,
                                   void *stream) {
    clear_error();
    if (!code || !llr || !synd || !target || !alpha || !beta || !grad_alpha || !grad_beta)
        QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    const CodeDev &d = code->d;
    qkdrec_status s = woms_check(d, F, T, ckpt_every, workspace);
    if (s != QKDREC_OK) return s;
    const WomsLayout l = woms_layout(d, F, T, ckpt_every);
    if (workspace_bytes < l.total) QKD_FAIL(QKDREC_ERR_ARG, "workspace %zu < %zu bytes", workspace_bytes, l.total);
    cudaStream_t st = as_stream(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    const int K = ckpt_every;
    const size_t me = (size_t)d.E * l.Fp, ve = (size_t)d.n * l.Fp;
    WomsArgs a = woms_args(d, F, alpha, beta, ws, l);
    a.gL = reinterpret_cast<float *>(ws + l.gL);
    a.gm = reinterpret_cast<float *>(ws + l.gm);
    float *mb = reinterpret_cast<float *>(ws + l.seg_m), *Lb = reinterpret_cast<float *>(ws + l.seg_L);
    // the checkpoints were written by qkdrec_woms_forward on this workspace; the
    // layout-converted inputs are rebuilt (the forward's ring reused seg_L[0])
    if ((s = woms_prepare(d, llr, synd, target, F, ws, l, st)) != QKDREC_OK) return s;
    QKD_CUDA(cudaMemsetAsync(ws + l.grads, 0, sizeof(double) * 4 * (size_t)T, st));
    QKD_CUDA(cudaMemsetAsync(ws + l.gm, 0, me * 4, st));
    const Geom g = check_geom(l.Fp, 1, d.M);
    const size_t stash = (size_t)kCheckWarps * kStash * 32 * sizeof(float);
    const unsigned vgrid = (unsigned)std::min<int64_t>(ceil_div((int64_t)d.n * l.Fp, 256), (int64_t)sm_count() * 32);
    for (int seg = l.nseg - 1; seg >= 0; --seg) {
        const int t0 = seg * K, t1 = std::min(t0 + K, (int)T);
        // m^{t0} and L^{t0} = llr + sum m^{t0}
        if (t0 == 0) {
            QKD_CUDA(cudaMemcpyAsync(Lb, ws + l.llr_i, ve * 4, cudaMemcpyDeviceToDevice, st));
        } else {
            QKD_CUDA(cudaMemcpyAsync(mb, ws + l.ckpt + (size_t)(seg - 1) * me * 4, me * 4,
                                     cudaMemcpyDeviceToDevice, st));
            a.m_out = mb;
            a.L_out = Lb;
            prof::Scope ps(prof::kWomsVar, st);
            woms_var_fwd<<<vgrid, 256, 0, st>>>(a);
        }
        woms_forward_range(a, d, l, ws, t0, t1, true, K, st);
        if (seg == l.nseg - 1) {
            a.L_in = Lb + ve * (t1 - t0);
            prof::Scope ps(prof::kFinish, st);
            QKD_CUDA(cudaMemsetAsync(ws + l.loss, 0, sizeof(double), st));
            woms_loss<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)d.n * l.Fp, 256), 4096), 256, 0, st>>>(a, 1);
        }
        for (int t = t1; t > t0; --t) {
            a.t = t;
            a.L_in = Lb + ve * (t - 1 - t0);
            a.m_in = (t == 1) ? nullptr : mb + me * (t - 1 - t0);
            a.prof = prof::counters(prof::kWomsBwd);
            {
                prof::Scope ps(prof::kWomsBwd, st);
                woms_check_bwd<<<g.grid, kCheckWarps * 32, stash, st>>>(a);
            }
            a.prof = prof::counters(prof::kWomsVar);
            {
                prof::Scope ps(prof::kWomsVar, st);
                woms_var_bwd<<<vgrid, 256, 0, st>>>(a);
            }
        }
        QKD_LAUNCHED("woms backward");
    }
    grads_out<<<(unsigned)ceil_div(2 * T, 128), 128, 0, st>>>(a.grads, T, grad_alpha, grad_beta);
    QKD_LAUNCHED("woms grads");
    return QKDREC_OK;
}

}  // extern "C"

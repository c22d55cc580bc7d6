// Layered offset min-sum (included by decode.cu).
//
// Layers are the greedy first-fit partition of the checks stored in the code
// object; inside a layer no two checks share a variable, so every check of a
// layer updates its posteriors in place without races:
//   q = L_v - m_cv,  m_cv = (-1)^{s_c} prod sgn(q) * max(min_{v'!=v}|q| - beta, 0),
//   L_v = q + m_cv.
// One kernel launch per layer; after the last layer a parity-only pass tests
// the syndrome of the hard decision, and a small kernel retires the frames
// whose test passed.  With one frame per lane (V = 1) the q values of a check
// stay in registers between the two passes; the V = 4 variant for degrees
// above the register cache reads them again and keeps retired frames frozen.

// ------------------------------------------------------------ float layered
// CACHED (degree <= kStash, one frame per lane): the q values of a check are
// kept in shared memory ([warp][edge][lane]) between the two passes.
template <typename MsgT, int V, bool CACHED>
__global__ void __launch_bounds__(kCheckWarps * 32, V == 1 ? 6 : 3)
layer_oms_f(DecArgs a, const int32_t *__restrict__ lchk, int32_t lbeg, int32_t lsize) {
    extern __shared__ float qstash[];  // [kCheckWarps][dstash][32]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw;
    const int slot = lane / fvw, lfv = lane - slot * fvw;
    float *L = reinterpret_cast<float *>(a.L);
    MsgT *msg = reinterpret_cast<MsgT *>(a.msg);
    const int64_t nvec = a.Fp / V;
    const uint32_t vmask = (1u << V) - 1u;
    constexpr int CH = V == 1 ? 4 : chunk_of<V>();   // 6 blocks per SM at one frame per lane
    constexpr int LG = lgfb_of<V>();
    constexpr bool STASH = CACHED && V == 1;
    float *my = qstash + (warp * a.dstash) * 32 + lane;
    unsigned long long units = 0;
    const int32_t nblk = *a.blk_n;
    for (int32_t bi = blockIdx.y; bi < nblk; bi += gridDim.y) {
        const int64_t fb = __ldg(a.blk + bi);
        const int64_t fv = fb * fvw + lfv, f0 = fv * V;
        if (fv >= nvec) continue;
        const int64_t bL = fpos(0, a.n, f0, LG), bM = fpos(0, a.E, f0, LG);  // item 0 of this lane
        const uint32_t act = active_bits<V>(a.active + f0);
        if (!act) continue;
        const int nact = __popc(act);
        const int64_t k0c = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
        for (int it = 0; it < kChecksPerWarp; ++it) {
            const int64_t kk = k0c + it * slots + slot;
            if (kk >= lsize) break;
            const int32_t c = __ldg(lchk + lbeg + kk);
            const int32_t beg = __ldg(a.rp + c), end = __ldg(a.rp + c + 1), d = end - beg;
            uint32_t neg = (__ldg(a.sbits + (int64_t)c * a.W + (f0 >> 5)) >> (f0 & 31)) & vmask;
            units += (unsigned long long)d * nact;
            float mn1[V], mn2[V];
            int32_t arg[V];
            for (int i = 0; i < V; ++i) { mn1[i] = INFINITY; mn2[i] = INFINITY; arg[i] = -1; }
            // pass 1: q = L - m on every edge (CH loads in flight, indices clamped)
            for (int k0 = 0; k0 < d; k0 += CH) {
                VF<V> Lv[CH], mo[CH];
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int kk = min(k0 + j, d - 1);
                    const int32_t e = beg + kk;
                    const int32_t col = __ldg(a.ci + e);
                    Lv[j] = ldf_plain<V>(L + bL + ((uint32_t)col << LG));
                    mo[j] = ldm<V>(msg + bM + ((uint32_t)(e) << LG));
                }
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int k = k0 + j;
                    if (k >= d) break;
                    for (int i = 0; i < V; ++i) {
                        const float q = Lv[j].v[i] - mo[j].v[i];
                        if (STASH) my[k * 32] = q;
                        neg ^= (uint32_t)(q < 0.0f) << i;
                        const float m = fabsf(q);
                        if (m < mn1[i]) { mn2[i] = mn1[i]; mn1[i] = m; arg[i] = k; }
                        else if (m < mn2[i]) mn2[i] = m;
                    }
                }
            }
            // pass 2: new messages and posteriors L = q + m
            for (int k = 0; k < d; ++k) {
                const int32_t e = beg + k;
                const int32_t col = __ldg(a.ci + e);
                float *Lp = L + bL + ((uint32_t)col << LG);
                MsgT *mp = msg + bM + ((uint32_t)(e) << LG);
                VF<V> q, Lold;
                if (STASH) {
                    q.v[0] = my[k * 32];
                } else {
                    Lold = ldf_plain<V>(Lp);
                    const VF<V> mo = ldm<V>(mp);
                    for (int i = 0; i < V; ++i) q.v[i] = Lold.v[i] - mo.v[i];
                }
                VF<V> mn, Ln;
                for (int i = 0; i < V; ++i) {
                    const float mag = fmaxf(((k == arg[i]) ? mn2[i] : mn1[i]) - a.beta, 0.0f);
                    mn.v[i] = (((neg >> i) & 1u) ^ (q.v[i] < 0.0f)) ? -mag : mag;
                    // later layers subtract the stored (possibly FP16-rounded) message;
                    // a retired frame keeps its posterior
                    Ln.v[i] = (STASH || ((act >> i) & 1u)) ? q.v[i] + as_stored(mn.v[i], msg) : Lold.v[i];
                }
                stm<V>(mp, mn);
                stf<V>(Lp, Ln);
            }
        }
    }
    // posterior read + written and message read + written, per active edge-frame
    prof_add(a.prof, units, units * (2 * sizeof(MsgT) + 8));
}

// ---------------------------------------------------------- integer layered
template <int V, bool CACHED>
__global__ void __launch_bounds__(kCheckWarps * 32, V == 1 ? 8 : 3)
layer_oms_i(DecArgs a, const int32_t *__restrict__ lchk, int32_t lbeg, int32_t lsize) {
    extern __shared__ float qstash[];  // [kCheckWarps][dstash][32], holds ints
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw;
    const int slot = lane / fvw, lfv = lane - slot * fvw;
    int16_t *L = reinterpret_cast<int16_t *>(a.L);
    int8_t *msg = reinterpret_cast<int8_t *>(a.msg);
    const int64_t nvec = a.Fp / V;
    const uint32_t vmask = (1u << V) - 1u;
    constexpr int CH = V == 1 ? 2 : chunk_of<V>();   // 8 blocks per SM at one frame per lane
    constexpr int LG = lgfb_of<V>();
    constexpr bool STASH = CACHED && V == 1;
    int *my = reinterpret_cast<int *>(qstash) + (warp * a.dstash) * 32 + lane;
    unsigned long long units = 0;
    const int32_t nblk = *a.blk_n;
    for (int32_t bi = blockIdx.y; bi < nblk; bi += gridDim.y) {
        const int64_t fb = __ldg(a.blk + bi);
        const int64_t fv = fb * fvw + lfv, f0 = fv * V;
        if (fv >= nvec) continue;
        const int64_t bL = fpos(0, a.n, f0, LG), bM = fpos(0, a.E, f0, LG);  // item 0 of this lane
        const uint32_t act = active_bits<V>(a.active + f0);
        if (!act) continue;
        const int nact = __popc(act);
        const int64_t k0c = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
        for (int it = 0; it < kChecksPerWarp; ++it) {
            const int64_t kk = k0c + it * slots + slot;
            if (kk >= lsize) break;
            const int32_t c = __ldg(lchk + lbeg + kk);
            const int32_t beg = __ldg(a.rp + c), end = __ldg(a.rp + c + 1), d = end - beg;
            uint32_t neg = (__ldg(a.sbits + (int64_t)c * a.W + (f0 >> 5)) >> (f0 & 31)) & vmask;
            units += (unsigned long long)d * nact;
            int mn1[V], mn2[V], arg[V];
            for (int i = 0; i < V; ++i) { mn1[i] = 1 << 20; mn2[i] = 1 << 20; arg[i] = -1; }
            // q_full = sat16(L - m); the v->c message is q_full clipped to 6 bits
            for (int k0 = 0; k0 < d; k0 += CH) {
                VI<V> Lv[CH], mo[CH];
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int32_t e = beg + min(k0 + j, d - 1);
                    Lv[j] = ldi16<V>(L + bL + ((uint32_t)__ldg(a.ci + e) << LG));
                    mo[j] = ldi8s<V>(msg + bM + ((uint32_t)(e) << LG));
                }
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    const int k = k0 + j;
                    if (k >= d) break;
                    for (int i = 0; i < V; ++i) {
                        const int qf = max(min(Lv[j].v[i] - mo[j].v[i], kPMax), -kPMax);
                        if (STASH) my[k * 32] = qf;
                        const int q = max(min(qf, kQMax), -kQMax);
                        neg ^= (uint32_t)(q < 0) << i;
                        const int m = q < 0 ? -q : q;
                        if (m < mn1[i]) { mn2[i] = mn1[i]; mn1[i] = m; arg[i] = k; }
                        else if (m < mn2[i]) mn2[i] = m;
                    }
                }
            }
            for (int k = 0; k < d; ++k) {
                const int32_t e = beg + k;
                int16_t *Lp = L + bL + ((uint32_t)__ldg(a.ci + e) << LG);
                int8_t *mp = msg + bM + ((uint32_t)(e) << LG);
                VI<V> qf, Lold;
                if (STASH) {
                    qf.v[0] = my[k * 32];
                } else {
                    Lold = ldi16<V>(Lp);
                    const VI<V> mo = ldi8s<V>(mp);
                    for (int i = 0; i < V; ++i) qf.v[i] = max(min(Lold.v[i] - mo.v[i], kPMax), -kPMax);
                }
                VI<V> mn, Ln;
                for (int i = 0; i < V; ++i) {
                    const int q = max(min(qf.v[i], kQMax), -kQMax);
                    const int mag = max(((k == arg[i]) ? mn2[i] : mn1[i]) - 1, 0);
                    mn.v[i] = (((neg >> i) & 1u) ^ (q < 0)) ? -mag : mag;
                    Ln.v[i] = (STASH || ((act >> i) & 1u)) ? max(min(qf.v[i] + mn.v[i], kPMax), -kPMax) : Lold.v[i];
                }
                sti8<V>(mp, mn);
                sti16<V>(Lp, Ln);
            }
        }
    }
    prof_add(a.prof, units, units * (2 * 1 + 2 * 2));
}

// Retire frames whose stopping test passed after iteration t (iters = t) and
// clear the other parity buffer for the next test.
__global__ void retire(int64_t Fp, int64_t W, int32_t t, uint8_t *active, int32_t *iters_i,
                       const uint32_t *__restrict__ unsat_cur, uint32_t *unsat_next) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f < W) unsat_next[f] = 0;
    if (f >= Fp) return;
    if (active[f] && !((unsat_cur[f >> 5] >> (f & 31)) & 1u)) {
        active[f] = 0;
        iters_i[f] = t;
    }
}

static void launch_layer(DecArgs a, const CodeDev &d, int prec, int32_t lb, int32_t ls, cudaStream_t st) {
    const int V = a.lgfb == lgfb_of<1>() ? 1 : 4;
    const Geom g = list_geom(a.Fp, V, ls);
    a.fvw = g.fvw;
    const dim3 B(kCheckWarps * 32);
    a.dstash = std::min(std::max(d.dc_max, 1), kStash);
    const size_t stash = (size_t)kCheckWarps * a.dstash * 32 * sizeof(float);
    const int32_t *lc = d.layer_chk;
    if (prec == kI8) {
        if (V == 1) layer_oms_i<1, true><<<g.grid, B, stash, st>>>(a, lc, lb, ls);
        else layer_oms_i<4, false><<<g.grid, B, 0, st>>>(a, lc, lb, ls);
    } else if (prec == kF16) {
        if (V == 1) layer_oms_f<__half, 1, true><<<g.grid, B, stash, st>>>(a, lc, lb, ls);
        else layer_oms_f<__half, 4, false><<<g.grid, B, 0, st>>>(a, lc, lb, ls);
    } else {
        if (V == 1) layer_oms_f<float, 1, true><<<g.grid, B, stash, st>>>(a, lc, lb, ls);
        else layer_oms_f<float, 4, false><<<g.grid, B, 0, st>>>(a, lc, lb, ls);
    }
}

#include "decode_qc.cuh"

// ------------------------------------------------- quasi-cyclic layer launch
__device__ int32_t g_qc_timeouts = 0;

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// checks per CTA chunk: two stages of (two posterior tiles per base column +
// one message tile) of Zc x 128 B each within ~96 KB (two CTAs per SM); the
// message tile's Zc nb rows within one tile copy (<= 256 rows)
static int qc_chunk(const CodeDev &d) {
    int zc = 256;
    while (zc > 1 && (zc > d.qc_Z || zc * d.qc_nb > 256 || (size_t)6 * d.qc_nb * zc * 128 > (size_t)96 * 1024))
        zc >>= 1;
    return zc;
}

static bool qc_usable(const CodeDev &d, int prec, int lgfb) {
    return d.qc_Z > 0 && d.qc_tma && prec == kF32 && lgfb == lgfb_of<1>() && encode_tiled() != nullptr;
}

// Tensor map of the messages [Fp/32][E][32], tiles of Zc nb edges.
static qkdrec_status qc_msg_map(const CodeDev &d, void *msg, int64_t Fp, CUtensorMap *tm) {
    const cuuint64_t dims[3] = {32, (cuuint64_t)d.E, (cuuint64_t)(Fp >> 5)};
    const cuuint64_t strides[2] = {32 * 4, (cuuint64_t)d.E * 128};
    const cuuint32_t box[3] = {32, (cuuint32_t)(qc_chunk(d) * d.qc_nb), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode_tiled()(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, msg, dims, strides, box, estr,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) QKD_FAIL(QKDREC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return QKDREC_OK;
}

// Tensor map of the posteriors [Fp/32][nb][Z][32] (one decode's workspace).
static qkdrec_status qc_tensor_map(const CodeDev &d, void *L, int64_t Fp, CUtensorMap *tm) {
    const cuuint64_t dims[4] = {32, (cuuint64_t)d.qc_Z, (cuuint64_t)d.qc_nb, (cuuint64_t)(Fp >> 5)};
    const cuuint64_t strides[3] = {32 * 4, (cuuint64_t)d.qc_Z * 128, (cuuint64_t)d.qc_nb * d.qc_Z * 128};
    const cuuint32_t box[4] = {32, (cuuint32_t)qc_chunk(d), 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode_tiled()(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, L, dims, strides, box, estr,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) QKD_FAIL(QKDREC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return QKDREC_OK;
}

static qkdrec_status launch_layer_qc(DecArgs a, const CodeDev &d, int32_t row, const CUtensorMap &tm,
                                     const CUtensorMap &tmm, cudaStream_t st) {
    static bool attr_set = false;
    const int zc = qc_chunk(d);
    const size_t smem = (size_t)6 * d.qc_nb * zc * 128 + 128;
    if (!attr_set) {
        QKD_CUDA(cudaFuncSetAttribute(layer_qc_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((size_t)96 * 1024 + 128)));
        attr_set = true;
    }
    QcLayer q;
    q.shift = d.qc_shift;
    q.Z = d.qc_Z;
    q.nb = d.qc_nb;
    q.row = row;
    q.Zc = zc;
    QKD_CUDA(cudaGetSymbolAddress(reinterpret_cast<void **>(&q.timeouts), g_qc_timeouts));
    const int64_t chunks = ceil_div(d.qc_Z, zc);
    const int64_t nblk = a.Fp >> 5;
    const int64_t gy = std::min<int64_t>(nblk, std::max<int64_t>(1, ceil_div((int64_t)sm_count() * 16, chunks)));
    layer_qc_tma<<<dim3((unsigned)chunks, (unsigned)std::min<int64_t>(gy, 65535)), 256, smem, st>>>(a, tm, tmm, q);
    QKD_LAUNCHED("layer_qc_tma");
    return QKDREC_OK;
}

qkdrec_status run_layered(const CodeDev &d, const float *llr, const SyndIn &synd, int32_t F,
                          const qkdrec_decode_opts &o, int prec, const uint8_t *conv_prev, bool compact,
                          uint8_t *bits_out, int32_t *iters_out, uint8_t *conv_out, float *post_out,
                          char *ws, cudaStream_t st) {
    const Layout l = make_layout(d, F, o.algo, prec);
    DecArgs a;
    Prepared pr;
    qkdrec_status s = prepare(d, llr, synd, F, o, prec, conv_prev, compact, ws, l, st, a, pr);
    if (s != QKDREC_OK) return s;
    const std::vector<int32_t> &lptr = d.h_layer_ptr;
    const int T = o.max_iter;
    auto parity = [&](int t) {
        DecArgs p = a;
        p.t = t;
        p.do_msgs = 0;
        p.early_stop = 1;
        p.unsat_cur = pr.unsat[t & 1];
        p.unsat_next = pr.unsat[(t + 1) & 1];
        const int kind = prec == kI8 ? prof::kParityI8 : prof::kParityF32;
        p.prof = prof::counters(kind);
        prof::Scope ps(kind, st);
        launch_check(p, d, QKDREC_OMS_FLOOD, prec, st);
    };
    auto retire_at = [&](int t) {
        prof::Scope ps(prof::kFinish, st);
        retire<<<(unsigned)ceil_div(std::max<int64_t>(l.Fp, l.W), 256), 256, 0, st>>>(
            l.Fp, l.W, t, a.active, a.iters_i, pr.unsat[t & 1], pr.unsat[(t + 1) & 1]);
        // frames retired now leave the block list
        rebuild_blocks(l, ws, st);
    };
    if (o.early_stop) {
        parity(0);
        retire_at(0);
        QKD_LAUNCHED("retire");
    }
    const int lkind = prec == kI8 ? prof::kLayerI8 : (prec == kF16 ? prof::kLayerF16 : prof::kLayerF32);
    // quasi-cyclic codes: posterior tiles staged by TMA (same results)
    const bool qc = qc_usable(d, prec, l.lgfb);
    CUtensorMap tm, tmm;
    if (qc && (s = qc_tensor_map(d, a.L, l.Fp, &tm)) != QKDREC_OK) return s;
    if (qc && (s = qc_msg_map(d, a.msg, l.Fp, &tmm)) != QKDREC_OK) return s;
    for (int t = 1; t <= T; ++t) {
        a.prof = prof::counters(qc ? prof::kLayerQc : lkind);
        for (int32_t ly = 0; ly < d.n_layers; ++ly) {
            prof::Scope ps(qc ? prof::kLayerQc : lkind, st);
            if (qc) {
                if ((s = launch_layer_qc(a, d, ly, tm, tmm, st)) != QKDREC_OK) return s;
            } else {
                launch_layer(a, d, prec, lptr[ly], lptr[ly + 1] - lptr[ly], st);
            }
        }
        QKD_LAUNCHED("layer_oms");
        if (o.early_stop) {
            parity(t);
            retire_at(t);
            QKD_LAUNCHED("retire");
        }
    }
    // final stopping test on the last posteriors: parity buffer (T+1)&1 is clear
    parity(T + 1);
    QKD_LAUNCHED("parity");
    return finish(d, F, T, prec, o, conv_prev, compact ? reinterpret_cast<const int32_t *>(ws + l.fmap) : nullptr,
                  compact ? reinterpret_cast<const int32_t *>(ws + l.fcnt) : nullptr, ws, l, pr, a, (T + 1) & 1,
                  bits_out, iters_out, conv_out, post_out, st);
}

// Layered offset min-sum (included by decode.cu).
//
// Layers are the greedy first-fit partition of the checks stored in the code
// object; inside a layer no two checks share a variable, so every check of a
// layer updates its posteriors in place without races:
//   q = L_v - m_cv,  m_cv = (-1)^{s_c} prod sgn(q) * max(min_{v'!=v}|q| - beta, 0),
//   L_v = q + m_cv.
// One kernel launch per layer; after the last layer a parity-only pass tests
// the syndrome of the hard decision, and a small kernel retires the frames
// whose test passed.

// ------------------------------------------------------------ float layered
template <typename MsgT>
__global__ void __launch_bounds__(kCheckWarps * 32)
layer_oms_f(DecArgs a, const int32_t *__restrict__ lchk, int32_t lbeg, int32_t lsize) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw;
    const int slot = lane / fvw, lfv = lane - slot * fvw;
    float *L = reinterpret_cast<float *>(a.L);
    MsgT *msg = reinterpret_cast<MsgT *>(a.msg);
    unsigned long long units = 0;
    for (int64_t fb = blockIdx.y; fb * fvw < a.FV; fb += gridDim.y) {
        const int64_t fv = fb * fvw + lfv;
        if (fv >= a.FV) continue;
        const uint32_t act = active4(a.active, fv);
        if (!act) continue;
        const int nact = __popc(act & 0x01010101u);
        const int64_t k0 = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
        for (int it = 0; it < kChecksPerWarp; ++it) {
            const int64_t k = k0 + it * slots + slot;
            if (k >= lsize) break;
            const int32_t c = __ldg(lchk + lbeg + k);
            const int32_t beg = __ldg(a.rp + c), end = __ldg(a.rp + c + 1);
            const uint32_t sw = __ldg(a.sbits + (int64_t)c * a.W + ((4 * fv) >> 5));
            uint32_t neg = (sw >> ((4 * fv) & 31)) & 0xfu;
            units += (unsigned long long)(end - beg) * nact;
            float mn1[4], mn2[4];
            int32_t arg[4];
            for (int i = 0; i < 4; ++i) { mn1[i] = INFINITY; mn2[i] = INFINITY; arg[i] = -1; }
            for (int32_t e = beg; e < end; ++e) {
                const int32_t v = __ldg(a.ci + e);
                const F4 Lv = *reinterpret_cast<const F4 *>(L + ((int64_t)v * a.FV + fv) * 4);
                const F4 mo = ld_msg(msg + ((int64_t)e * a.FV + fv) * 4);
                for (int i = 0; i < 4; ++i) {
                    const float q = Lv.v[i] - mo.v[i];
                    neg ^= (uint32_t)(q < 0.0f) << i;
                    const float m = fabsf(q);
                    if (m < mn1[i]) { mn2[i] = mn1[i]; mn1[i] = m; arg[i] = e; }
                    else if (m < mn2[i]) mn2[i] = m;
                }
            }
            for (int32_t e = beg; e < end; ++e) {
                const int32_t v = __ldg(a.ci + e);
                float *Lp = L + ((int64_t)v * a.FV + fv) * 4;
                const F4 Lv = *reinterpret_cast<const F4 *>(Lp);
                MsgT *mp = msg + ((int64_t)e * a.FV + fv) * 4;
                const F4 mo = ld_msg(mp);
                F4 mn, Ln;
                for (int i = 0; i < 4; ++i) {
                    const float q = Lv.v[i] - mo.v[i];
                    const bool sneg = ((neg >> i) & 1u) ^ (q < 0.0f);
                    const float mag = fmaxf(((e == arg[i]) ? mn2[i] : mn1[i]) - a.beta, 0.0f);
                    mn.v[i] = sneg ? -mag : mag;
                }
                st_msg(mp, mn);
                // the stored (possibly FP16-rounded) message is what later layers subtract
                const F4 ms = as_stored<MsgT>(mn);
                for (int i = 0; i < 4; ++i) {
                    const float q = Lv.v[i] - mo.v[i];
                    Ln.v[i] = act_bit(act, i) ? q + ms.v[i] : Lv.v[i];
                }
                st_f4(Lp, Ln);
            }
        }
    }
    // posterior read + written and message read + written, per active edge-frame
    prof_add(a.prof, units, units * (2 * sizeof(MsgT) + 8));
}

// ---------------------------------------------------------- integer layered
__global__ void __launch_bounds__(kCheckWarps * 32)
layer_oms_i(DecArgs a, const int32_t *__restrict__ lchk, int32_t lbeg, int32_t lsize) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int fvw = a.fvw, slots = 32 / fvw;
    const int slot = lane / fvw, lfv = lane - slot * fvw;
    int16_t *L = reinterpret_cast<int16_t *>(a.L);
    int8_t *msg = reinterpret_cast<int8_t *>(a.msg);
    unsigned long long units = 0;
    for (int64_t fb = blockIdx.y; fb * fvw < a.FV; fb += gridDim.y) {
        const int64_t fv = fb * fvw + lfv;
        if (fv >= a.FV) continue;
        const uint32_t act = active4(a.active, fv);
        if (!act) continue;
        const int nact = __popc(act & 0x01010101u);
        const int64_t k0 = ((int64_t)blockIdx.x * kCheckWarps + warp) * (kChecksPerWarp * slots);
        for (int it = 0; it < kChecksPerWarp; ++it) {
            const int64_t k = k0 + it * slots + slot;
            if (k >= lsize) break;
            const int32_t c = __ldg(lchk + lbeg + k);
            const int32_t beg = __ldg(a.rp + c), end = __ldg(a.rp + c + 1);
            const uint32_t sw = __ldg(a.sbits + (int64_t)c * a.W + ((4 * fv) >> 5));
            uint32_t neg = (sw >> ((4 * fv) & 31)) & 0xfu;
            units += (unsigned long long)(end - beg) * nact;
            int mn1[4], mn2[4], arg[4];
            for (int i = 0; i < 4; ++i) { mn1[i] = 1 << 20; mn2[i] = 1 << 20; arg[i] = -1; }
            for (int32_t e = beg; e < end; ++e) {
                const int32_t v = __ldg(a.ci + e);
                const short4 l4 = *reinterpret_cast<const short4 *>(L + ((int64_t)v * a.FV + fv) * 4);
                const int Lv[4] = {l4.x, l4.y, l4.z, l4.w};
                const I4 mo = ld_i8x4(msg + ((int64_t)e * a.FV + fv) * 4);
                for (int i = 0; i < 4; ++i) {
                    const int qf = max(min(Lv[i] - mo.v[i], kPMax), -kPMax);
                    const int q = max(min(qf, kQMax), -kQMax);
                    neg ^= (uint32_t)(q < 0) << i;
                    const int m = q < 0 ? -q : q;
                    if (m < mn1[i]) { mn2[i] = mn1[i]; mn1[i] = m; arg[i] = e; }
                    else if (m < mn2[i]) mn2[i] = m;
                }
            }
            for (int32_t e = beg; e < end; ++e) {
                const int32_t v = __ldg(a.ci + e);
                int16_t *Lp = L + ((int64_t)v * a.FV + fv) * 4;
                const short4 l4 = *reinterpret_cast<const short4 *>(Lp);
                const int Lv[4] = {l4.x, l4.y, l4.z, l4.w};
                int8_t *mp = msg + ((int64_t)e * a.FV + fv) * 4;
                const I4 mo = ld_i8x4(mp);
                I4 mn, Ln;
                for (int i = 0; i < 4; ++i) {
                    const int qf = max(min(Lv[i] - mo.v[i], kPMax), -kPMax);
                    const int q = max(min(qf, kQMax), -kQMax);
                    const bool sneg = ((neg >> i) & 1u) ^ (q < 0);
                    const int mag = max(((e == arg[i]) ? mn2[i] : mn1[i]) - 1, 0);
                    mn.v[i] = sneg ? -mag : mag;
                    Ln.v[i] = act_bit(act, i) ? max(min(qf + mn.v[i], kPMax), -kPMax) : Lv[i];
                }
                st_i8x4(mp, mn);
                st_i16x4(Lp, Ln);
            }
        }
    }
    prof_add(a.prof, units, units * (2 * 1 + 2 * 2));
}

// Retire frames whose stopping test passed after iteration t (iters = t) and
// clear the other parity buffer for the next test.
__global__ void retire(int64_t Fp, int32_t t, uint8_t *active, int32_t *iters_i,
                       const uint32_t *__restrict__ unsat_cur, uint32_t *unsat_next) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= Fp) return;
    if (active[f] && !((unsat_cur[f >> 2] >> (f & 3)) & 1u)) {
        active[f] = 0;
        iters_i[f] = t;
    }
    if ((f & 3) == 0) unsat_next[f >> 2] = 0;
}

qkdrec_status run_layered(const CodeDev &d, const float *llr, const uint8_t *synd, int32_t F,
                          const qkdrec_decode_opts &o, int prec, const uint8_t *conv_prev,
                          uint8_t *bits_out, int32_t *iters_out, uint8_t *conv_out, float *post_out,
                          char *ws, cudaStream_t st) {
    const Layout l = make_layout(d, F, prec);
    DecArgs a;
    Prepared pr;
    qkdrec_status s = prepare(d, llr, synd, F, o, prec, conv_prev, ws, l, st, a, pr);
    if (s != QKDREC_OK) return s;
    const int slots = 32 / a.fvw;
    const int64_t checks_per_block = (int64_t)kCheckWarps * kChecksPerWarp * slots;
    const int64_t fblocks = ceil_div(l.FV, a.fvw);
    const unsigned gy = (unsigned)(fblocks < 65535 ? fblocks : 65535);
    const std::vector<int32_t> &lptr = d.h_layer_ptr;
    const int T = o.max_iter;
    auto parity = [&](int t) {
        a.t = t;
        a.do_msgs = 0;
        a.early_stop = 1;
        a.unsat_cur = pr.unsat[t & 1];
        a.unsat_next = pr.unsat[(t + 1) & 1];
        const int kind = prec == kI8 ? prof::kParityI8 : prof::kParityF32;
        a.prof = prof::counters(kind);
        prof::Scope ps(kind, st);
        dim3 cgrid((unsigned)ceil_div(d.M, checks_per_block), gy);
        if (prec == kI8) check_flood_i<true><<<cgrid, kCheckWarps * 32, 0, st>>>(a);
        else if (prec == kF16) check_flood_f<kOMS, __half><<<cgrid, kCheckWarps * 32, 0, st>>>(a);
        else check_flood_f<kOMS, float><<<cgrid, kCheckWarps * 32, 0, st>>>(a);
    };
    auto retire_at = [&](int t) {
        prof::Scope ps(prof::kFinish, st);
        retire<<<(unsigned)ceil_div(l.Fp, 256), 256, 0, st>>>(l.Fp, t, a.active, a.iters_i, pr.unsat[t & 1],
                                                             pr.unsat[(t + 1) & 1]);
    };
    if (o.early_stop) {
        parity(0);
        retire_at(0);
        QKD_LAUNCHED("retire");
    }
    for (int t = 1; t <= T; ++t) {
        const int lkind = prec == kI8 ? prof::kLayerI8 : (prec == kF16 ? prof::kLayerF16 : prof::kLayerF32);
        a.prof = prof::counters(lkind);
        for (int32_t ly = 0; ly < d.n_layers; ++ly) {
            prof::Scope ps(lkind, st);
            const int32_t lb = lptr[ly], ls = lptr[ly + 1] - lptr[ly];
            dim3 g((unsigned)ceil_div(ls, checks_per_block), gy);
            if (prec == kI8) layer_oms_i<<<g, kCheckWarps * 32, 0, st>>>(a, d.layer_chk, lb, ls);
            else if (prec == kF16) layer_oms_f<__half><<<g, kCheckWarps * 32, 0, st>>>(a, d.layer_chk, lb, ls);
            else layer_oms_f<float><<<g, kCheckWarps * 32, 0, st>>>(a, d.layer_chk, lb, ls);
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
    return finish(d, F, T, prec, o, conv_prev, ws, l, pr, a, (T + 1) & 1, bits_out, iters_out, conv_out,
                  post_out, st);
}

// Batched decoding of an uneven batch: many groups of frames, each group with
// its own code (length n, rate), in one persistent launch (included by decode.cu).
//
// The batch is cut into work items (group, tile of FT frames), ordered longest
// first.  A tile is decoded by a thread-block cluster of CS CTAs (CS = 1: one
// CTA): the cluster's leader takes the next item with one atomic increment of
// a queue head and hands it to the other CTAs through distributed shared
// memory; clusters never wait for each other.  The CTAs of the cluster split
// every layer's checks between their warps and meet at the hardware cluster
// barrier (release/acquire) after each layer, so one tile runs on up to 8 SMs:
// the tile that holds the batch's slowest frame (the one that needs every
// iteration) finishes up to 8 times sooner.  The cluster runs the whole layered
// offset min-sum decode of its tile: all layers of all iterations, the
// stopping test after every iteration (per-CTA partial results OR-ed into the
// leader's shared words, one per tile), frames retiring one by one, the tile leaving early
// once all its frames are done.
//
// Lane layout: a lane updates V consecutive frames (V = 1, 2 or 4) and FT / V
// lanes serve one check, lane = slot * (FT / V) + frame / V, so a warp serves
// 32 V / FT checks at a time; with FT / V = 8 lanes of 4 frames (or 32 lanes of
// one) every posterior gather and message access of a check is one 128-byte
// line.  Per tile the workspace holds L [n][FT] and m [E][FT] (frame fastest),
// the tile's syndrome bits (one word per check) and its hard decisions (one
// word per variable, bit f = L[v][f] < 0, flipped by an atomic XOR whenever an
// update changes a posterior's sign, so the stopping test XORs words instead of
// gathering posteriors).  Messages are not cleared: the first iteration reads
// m = 0 without loading it.  The q values of the first min(SF / V, 32) edges
// of a check (SF: floats of stash per lane) wait in shared memory between the
// two passes; the rest are recomputed from L and m, which no other check of
// the layer touches.  Once at most `sparse` frames of an item are decoding,
// the item switches to a mode with 8 lanes per (check, frame) (plan_item).  Posteriors go through L2 only (ld/st .cg), so what one SM of
// the cluster wrote is what the others read; messages stream with the
// evict-first hint (each check, hence each message, is always handled by the
// same warp of the same CTA), so L2 keeps the tiles' posteriors, which the
// checks gather.

namespace qkd {
namespace cg = cooperative_groups;

struct PlanGroup {
    const int32_t *rp, *ci, *lptr, *lchk;
    const float *llr;       // [F][n]
    const uint8_t *synd;    // [F][M]
    uint8_t *bits;          // [F][n]
    int32_t *iters;         // [F]
    uint8_t *conv;          // [F]
    int64_t ws_off;         // byte offset of the group's first tile
    int64_t tile_bytes;
    int64_t E;
    int32_t n, M, n_layers, F, dc_max;
};

struct PlanItem {
    int32_t g, tile, ntiles;   // tiles tile .. tile + ntiles - 1 of group g, decoded together
};

constexpr int kPlanMaxTiles = 4;   // tiles of one work item
constexpr int kPlanMaxSparse = 32; // sparse mode serves at most this many frames of an item

// dynamic shared memory per warp: the q stash / transpose area
// floats of q stash per lane for a launch variant of at most NT threads: the
// stash is NT * SF * 4 = 128 KB per CTA in every variant (one CTA per SM)
__host__ __device__ constexpr int plan_stash_floats(int NT) { return NT >= 1024 ? 32 : (NT >= 512 ? 64 : 128); }

struct PlanArgs {
    const PlanGroup *groups;
    const PlanItem *items;
    int32_t n_items;
    int32_t *head;
    char *ws;
    int32_t FT, CS, max_iter, early_stop;
    int32_t sparse;   // items with at most this many decoding frames run in sparse mode
    float beta;
    unsigned long long *prof;
};

// A tile: L [n][FT], m [E][FT], the syndrome bits [M] (one word per check,
// bit f = frame f) and the hard decisions [n] (bit f of word v = L[v][f] < 0).
static int64_t plan_tile_bytes(int64_t n, int64_t E, int64_t M, int FT) {
    return (int64_t)align_up((size_t)n * FT * 4, 256) + (int64_t)align_up((size_t)E * FT * 4, 256) +
           (int64_t)align_up((size_t)M * 4, 256) + (int64_t)align_up((size_t)n * 4, 256);
}

// barrier over the CTAs that share a tile
__device__ __forceinline__ void plan_sync(int CS) {
    if (CS > 1) cg::this_cluster().sync();
    else __syncthreads();
}

// V consecutive frames of one lane (V = 1, 2 or 4): posteriors through L2
// only (.cg), messages streamed (.cs), q values in this warp's shared stash.
template <int V> __device__ __forceinline__ VF<V> pl_ld_L(const float *p) {
    if constexpr (V == 1) {
        return VF<1>{{__ldcg(p)}};
    } else if constexpr (V == 2) {
        const float2 t = __ldcg(reinterpret_cast<const float2 *>(p));
        return VF<2>{{t.x, t.y}};
    } else {
        const float4 t = __ldcg(reinterpret_cast<const float4 *>(p));
        return VF<4>{{t.x, t.y, t.z, t.w}};
    }
}
template <int V> __device__ __forceinline__ VF<V> pl_ld_m(const float *p) {
    if constexpr (V == 1) {
        return VF<1>{{__ldcs(p)}};
    } else if constexpr (V == 2) {
        const float2 t = __ldcs(reinterpret_cast<const float2 *>(p));
        return VF<2>{{t.x, t.y}};
    } else {
        const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
        return VF<4>{{t.x, t.y, t.z, t.w}};
    }
}
// Stores of the frames set in `live` (a retired frame keeps its values): one
// vector store when all V are live.
template <int V> __device__ __forceinline__ void pl_st_L(float *p, const VF<V> &a, uint32_t live) {
    if constexpr (V == 1) {
        __stcg(p, a.v[0]);
    } else if (live == (1u << V) - 1u) {
        if constexpr (V == 2) __stcg(reinterpret_cast<float2 *>(p), make_float2(a.v[0], a.v[1]));
        else __stcg(reinterpret_cast<float4 *>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i)
            if ((live >> i) & 1u) __stcg(p + i, a.v[i]);
    }
}
template <int V> __device__ __forceinline__ void pl_st_m(float *p, const VF<V> &a, uint32_t live) {
    if constexpr (V == 1) {
        __stcs(p, a.v[0]);
    } else if (live == (1u << V) - 1u) {
        if constexpr (V == 2) __stcs(reinterpret_cast<float2 *>(p), make_float2(a.v[0], a.v[1]));
        else __stcs(reinterpret_cast<float4 *>(p), make_float4(a.v[0], a.v[1], a.v[2], a.v[3]));
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i)
            if ((live >> i) & 1u) __stcs(p + i, a.v[i]);
    }
}
template <int V> __device__ __forceinline__ void pl_st_sh(float *p, const VF<V> &a) {
    if constexpr (V == 1) *p = a.v[0];
    else if constexpr (V == 2) *reinterpret_cast<float2 *>(p) = make_float2(a.v[0], a.v[1]);
    else *reinterpret_cast<float4 *>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
template <int V> __device__ __forceinline__ VF<V> pl_ld_sh(const float *p) {
    if constexpr (V == 1) {
        return VF<1>{{*p}};
    } else if constexpr (V == 2) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        return VF<2>{{t.x, t.y}};
    } else {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        return VF<4>{{t.x, t.y, t.z, t.w}};
    }
}

// One check's layered update for the V frames a lane holds (live: the frames
// of those V still decoding; L, msg point at the lane's first frame f_lo of
// the tile, whose rows are FT floats apart; st: the lane's stash, edge kq at
// st[kq * 32 * V]; neg: the check's syndrome bits of the V frames; hd: the
// tile's hard-decision words, whose bits of the frames whose sign changes
// are flipped):
//   pass 1: q = L - m on every edge (CH loads in flight, indices clamped),
//           sign parity and the two smallest |q| per frame;
//   pass 2: m' = sign * max(min_{other edges} |q| - beta, 0), L = q + m'.
// Edges beyond the stash get q again from L and m, which no other check of
// the layer touches.  The first iteration reads no message (m = 0).
template <int V, int CH, int SF>
__device__ __forceinline__ void plan_check(const int32_t *__restrict__ ci, int32_t beg, int32_t d, bool first,
                                           float *L, float *msg, int FT, uint32_t neg, uint32_t live, float *st,
                                           float beta, uint32_t *hd, int f_lo) {
    // stashed edges: SF / V, at most 32 (their old signs are bits of one word per frame)
    constexpr int SV = SF / V < 32 ? SF / V : 32;
    float mn1[V], mn2[V];
    int32_t arg[V];
    uint32_t ob[V];   // sign of the old posterior of each stashed edge (bit kq)
#pragma unroll
    for (int i = 0; i < V; ++i) {
        mn1[i] = INFINITY;
        mn2[i] = INFINITY;
        arg[i] = -1;
        ob[i] = 0;
    }
    for (int k0 = 0; k0 < d; k0 += CH) {
        VF<V> Lv[CH], mo[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int32_t e = beg + min(k0 + j, d - 1);
            Lv[j] = pl_ld_L<V>(L + (uint32_t)__ldg(ci + e) * FT);
            mo[j] = first ? VF<V>{} : pl_ld_m<V>(msg + (uint32_t)e * FT);
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int kq = k0 + j;
            if (kq >= d) break;
            VF<V> q;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                q.v[i] = Lv[j].v[i] - mo[j].v[i];
                if (kq < SV) ob[i] |= (uint32_t)(Lv[j].v[i] < 0.0f) << kq;
                neg ^= (uint32_t)(q.v[i] < 0.0f) << i;
                const float m = fabsf(q.v[i]);
                if (m < mn1[i]) {
                    mn2[i] = mn1[i];
                    mn1[i] = m;
                    arg[i] = kq;
                } else if (m < mn2[i]) {
                    mn2[i] = m;
                }
            }
            if (kq < SV) pl_st_sh<V>(st + kq * 32 * V, q);
        }
    }
    // oldneg: bit i = the old posterior of frame i was negative
    auto update = [&](int kq, const VF<V> &q, uint32_t col, float *mp, uint32_t oldneg) {
        VF<V> mo, lo;
        uint32_t flip = 0;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const float mag = fmaxf(((kq == arg[i]) ? mn2[i] : mn1[i]) - beta, 0.0f);
            mo.v[i] = (((neg >> i) ^ (uint32_t)(q.v[i] < 0.0f)) & 1u) ? -mag : mag;
            lo.v[i] = q.v[i] + mo.v[i];
            flip |= ((uint32_t)(lo.v[i] < 0.0f) ^ ((oldneg >> i) & 1u)) << i;
        }
        pl_st_m<V>(mp, mo, live);
        pl_st_L<V>(L + col * FT, lo, live);
        flip &= live;
        if (flip) atomicXor(hd + col, flip << f_lo);
    };
    // stashed edges: their column indices again, CH loads in flight
    const int ds = min(d, SV);
    for (int k0 = 0; k0 < ds; k0 += CH) {
        uint32_t col[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) col[j] = (uint32_t)__ldg(ci + beg + min(k0 + j, ds - 1));
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int kq = k0 + j;
            if (kq >= ds) break;
            uint32_t on = 0;
#pragma unroll
            for (int i = 0; i < V; ++i) on |= ((ob[i] >> kq) & 1u) << i;
            update(kq, pl_ld_sh<V>(st + kq * 32 * V), col[j], msg + (uint32_t)(beg + kq) * FT, on);
        }
    }
    for (int k0 = ds; k0 < d; k0 += CH) {
        VF<V> Lv[CH], mv[CH];
        uint32_t col[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int32_t e = beg + min(k0 + j, d - 1);
            col[j] = (uint32_t)__ldg(ci + e);
            Lv[j] = pl_ld_L<V>(L + col[j] * FT);
            mv[j] = first ? VF<V>{} : pl_ld_m<V>(msg + (uint32_t)e * FT);
        }
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            const int kq = k0 + j;
            if (kq >= d) break;
            VF<V> q;
            uint32_t on = 0;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                q.v[i] = Lv[j].v[i] - mv[j].v[i];
                on |= (uint32_t)(Lv[j].v[i] < 0.0f) << i;
            }
            update(kq, q, col[j], msg + (uint32_t)(beg + kq) * FT, on);
        }
    }
}

// Sparse mode: one (check, frame) task per kSG lanes, lane g of the task
// holding edges g, g + kSG, ... (SE of them in registers per pass segment:
// 4 or 8, so checks of up to 32 or 64 edges take one segment).
constexpr int kSG = 8;

// Merge of two lanes' (smallest |q|, second smallest, edge of the smallest,
// sign parity) over disjoint edge sets: on equal smallest values the lower edge
// index wins, as in one pass over the edges in order with strict comparisons.
__device__ __forceinline__ void plan_minmerge(float &mn1, float &mn2, int &arg, uint32_t &neg) {
#pragma unroll
    for (int o = 1; o < kSG; o <<= 1) {
        const float b1 = __shfl_xor_sync(0xffffffffu, mn1, o);
        const float b2 = __shfl_xor_sync(0xffffffffu, mn2, o);
        const int ba = __shfl_xor_sync(0xffffffffu, arg, o);
        neg ^= __shfl_xor_sync(0xffffffffu, neg, o);
        const bool take_b = b1 < mn1 || (b1 == mn1 && ba < arg);
        mn2 = fminf(fmaxf(mn1, b1), fminf(mn2, b2));
        mn1 = fminf(mn1, b1);
        arg = take_b ? ba : arg;
    }
}

// One check's layered update for one frame by the kSG lanes of a task (all 32
// lanes of the warp call it; live = this lane's task exists; g = lane within
// the task; neg0 = the check's syndrome bit).  The same rule as plan_check:
// the smallest and second smallest |q| and the sign parity over all edges,
// then m' = sign * max(min_{other edges} |q| - beta, 0) and L = q + m'.
template <int kSE>
__device__ __forceinline__ void plan_check_task(const int32_t *__restrict__ ci, int32_t beg, int32_t d, bool first,
                                                float *L, float *msg, int FT, uint32_t neg0, bool live, int g,
                                                float beta, uint32_t *hd, int f) {
    float q[kSE];
    uint32_t col[kSE], ob = 0;   // ob bit j: the old posterior of segment-0 edge j was negative
    float mn1 = INFINITY, mn2 = INFINITY;
    int arg = 0x7fffffff;
    uint32_t neg = g == 0 ? neg0 : 0u;
    const int dd = live ? d : 0;
    for (int base = 0; base < dd; base += kSG * kSE) {
        float Lv[kSE], mv[kSE];
        uint32_t cc[kSE];
#pragma unroll
        for (int j = 0; j < kSE; ++j) cc[j] = (uint32_t)__ldg(ci + beg + min(base + g + j * kSG, dd - 1));
#pragma unroll
        for (int j = 0; j < kSE; ++j) {
            const int kc = min(base + g + j * kSG, dd - 1);
            Lv[j] = __ldcg(L + cc[j] * FT);
            mv[j] = first ? 0.0f : __ldcs(msg + (uint32_t)(beg + kc) * FT);
        }
#pragma unroll
        for (int j = 0; j < kSE; ++j) {
            const int kq = base + g + j * kSG;
            const float qq = Lv[j] - mv[j];
            if (base == 0) {
                q[j] = qq;
                col[j] = cc[j];
                ob |= (uint32_t)(Lv[j] < 0.0f) << j;
            }
            if (kq < dd) {
                neg ^= (uint32_t)(qq < 0.0f);
                const float m = fabsf(qq);
                if (m < mn1) {
                    mn2 = mn1;
                    mn1 = m;
                    arg = kq;
                } else if (m < mn2) {
                    mn2 = m;
                }
            }
        }
    }
    plan_minmerge(mn1, mn2, arg, neg);
    for (int base = 0; base < dd; base += kSG * kSE) {
        float Lv[kSE], mv[kSE];
        uint32_t cc[kSE];
        if (base > 0) {   // edges beyond the first segment: q again from the unchanged L and m
#pragma unroll
            for (int j = 0; j < kSE; ++j) cc[j] = (uint32_t)__ldg(ci + beg + min(base + g + j * kSG, dd - 1));
#pragma unroll
            for (int j = 0; j < kSE; ++j) {
                const int kc = min(base + g + j * kSG, dd - 1);
                Lv[j] = __ldcg(L + cc[j] * FT);
                mv[j] = first ? 0.0f : __ldcs(msg + (uint32_t)(beg + kc) * FT);
            }
        }
#pragma unroll
        for (int j = 0; j < kSE; ++j) {
            const int kq = base + g + j * kSG;
            if (kq >= dd) break;
            const float qq = base == 0 ? q[j] : Lv[j] - mv[j];
            const uint32_t cj = base == 0 ? col[j] : cc[j];
            const uint32_t on = base == 0 ? (ob >> j) & 1u : (uint32_t)(Lv[j] < 0.0f);
            const float mag = fmaxf(((kq == arg) ? mn2 : mn1) - beta, 0.0f);
            const float mo = ((neg ^ (uint32_t)(qq < 0.0f)) & 1u) ? -mag : mag;
            const float ln = qq + mo;
            __stcs(msg + (uint32_t)(beg + kq) * FT, mo);
            __stcg(L + cj * FT, ln);
            if ((uint32_t)(ln < 0.0f) != on) atomicXor(hd + cj, 1u << f);
        }
    }
}

// Syndrome test of one check for all frames of a tile at once: the check's
// syndrome word XOR the hard-decision words of its variables (CH loads in
// flight); bit f of the result is set iff frame f fails the check.
template <int CH>
__device__ __forceinline__ uint32_t plan_parity_word(const int32_t *__restrict__ ci, int32_t beg, int32_t d,
                                                     const uint32_t *hd, uint32_t w) {
    for (int k0 = 0; k0 < d; k0 += CH) {
        uint32_t h[CH];
#pragma unroll
        for (int j = 0; j < CH; ++j) h[j] = __ldcg(hd + __ldg(ci + beg + min(k0 + j, d - 1)));
#pragma unroll
        for (int j = 0; j < CH; ++j)
            if (k0 + j < d) w ^= h[j];
    }
    return w;
}

// Per-launch work counters of one CTA.
struct PlanCount {
    unsigned long long units = 0, units_first = 0, pwords = 0;
};

// Decode one work item -- K tiles of one group -- with a team of tcs CTAs
// (trank = this CTA's place in the team; unsat_dst = the team leader's shared
// stopping-test words, one per tile).  The K tiles run their layers in step:
// between two barriers every warp handles its checks of the layer for each
// tile in turn, so a layer with few checks still gives the team K times the
// work per barrier.  Dense mode: each lane updates V consecutive frames of a
// tile with V-wide loads and stores, FT / V lanes serving one check.  Sparse
// mode, once at most a.sparse frames of the item are still decoding (the tail
// of a batch is the few frames that need many iterations): each lane serves
// one (check, decoding frame) pair with V * CH loads in flight, so a layer's
// checks spread over 32 / A times as many lanes and a layer costs about one
// check's chain of loads.  Every frame's arithmetic is the same in both modes.
template <int CH, int V, int SE, int SF>
__device__ __forceinline__ void plan_item(const PlanArgs &a, int item, int tcs, int trank, uint32_t *unsat_dst,
                                          uint32_t *s_unsat, float *qst, uint8_t *s_pair, PlanCount &cnt) {
    constexpr uint32_t vmask = (1u << V) - 1u;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int FT = a.FT, FL = FT / V, slots = 32 / FL, slot = lane / FL, fl = lane - slot * FL;
    const int f_lo = fl * V;                         // this lane's first frame in the tile
    // warp within the team, interleaved over the team's CTAs (SMs): a layer
    // with few checks still spreads over every SM of the team
    const int gw = warp * tcs + trank, TW = tcs * nwarps;
    const int64_t gt = (int64_t)trank * blockDim.x + tid, TT = (int64_t)tcs * blockDim.x;
    float *tr = qst + (warp * SF) * 32;              // this warp's 32 x SF floats (32 x 32 for transposes)
    uint32_t units = 0, units_first = 0, pwords = 0;   // this item's share (added to cnt at the end)
    const PlanItem itm = a.items[item];
    const PlanGroup &G = a.groups[itm.g];
    const int n = G.n, M = G.M, K = itm.ntiles;
    int f0[kPlanMaxTiles], nf[kPlanMaxTiles];
    float *Lt[kPlanMaxTiles], *mt[kPlanMaxTiles];
    uint32_t *swt[kPlanMaxTiles], *hdt[kPlanMaxTiles], active[kPlanMaxTiles];   // active: same in every thread
#pragma unroll
    for (int k = 0; k < kPlanMaxTiles; ++k) {
        const int tile = itm.tile + min(k, K - 1);
        f0[k] = tile * FT;
        nf[k] = k < K ? min(FT, G.F - f0[k]) : 0;
        char *tb = a.ws + G.ws_off + (int64_t)tile * G.tile_bytes;
        Lt[k] = reinterpret_cast<float *>(tb);
        mt[k] = reinterpret_cast<float *>(tb + align_up((size_t)n * FT * 4, 256));
        swt[k] = reinterpret_cast<uint32_t *>(tb + align_up((size_t)n * FT * 4, 256) + align_up((size_t)G.E * FT * 4, 256));
        hdt[k] = swt[k] + align_up((size_t)M * 4, 256) / 4;
        active[k] = nf[k] == 32 ? 0xffffffffu : ((1u << nf[k]) - 1u);
    }
    // ---- load the tiles: L[v][i] = llr[f0 + i][v] through a per-warp transpose
    // (swizzled columns, conflict-free), padding frames get a confident 0;
    // eight rows in flight per lane; the hard-decision word of each variable
    for (int k = 0; k < K; ++k) {
        float *L = Lt[k];
        for (int64_t v0 = (int64_t)gw * 32; v0 < n; v0 += (int64_t)TW * 32) {
            const int64_t v = v0 + lane;
            uint32_t hw = 0;
            for (int i0 = 0; i0 < FT; i0 += 8) {
                float t[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + u;
                    t[u] = (i < nf[k] && v < n) ? __ldg(G.llr + (int64_t)(f0[k] + i) * n + v) : kLlrClip;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    tr[(i0 + u) * 32 + (lane ^ (i0 + u))] = t[u];
                    hw |= (uint32_t)(t[u] < 0.0f) << (i0 + u);
                }
            }
            if (v < n) __stcg(hdt[k] + v, hw);
            __syncwarp();
            for (int idx = lane; idx < 32 * FT; idx += 32) {
                const int j = idx / FT, fi = idx - j * FT;
                if (v0 + j < n) __stcg(L + (v0 + j) * FT + fi, tr[fi * 32 + (j ^ fi)]);
            }
            __syncwarp();
        }
        for (int64_t c = gt; c < M; c += TT) {
            uint32_t w = 0;
#pragma unroll 8
            for (int i = 0; i < nf[k]; ++i) w |= (uint32_t)(__ldg(G.synd + (int64_t)(f0[k] + i) * M + c) & 1) << i;
            __stcg(swt[k] + c, w);
        }
    }
    plan_sync(tcs);
    // ---- sparse mode: A = frames of the item still decoding, listed in
    // s_pair as (tile << 5 | frame); task t of a layer = (check lb + t / A,
    // frame t mod A), kSG lanes per task, 32 / kSG tasks per warp
    int sA = 0;
    bool sparse = false;
    const int sg = lane & (kSG - 1), stask = lane / kSG;
    auto sparse_setup = [&]() {
        sA = 0;
        for (int k = 0; k < K; ++k) sA += __popc(active[k]);
        sparse = sA > 0 && sA <= a.sparse;
        if (!sparse) return;
        if (tid < sA) {
            int r = tid;
            for (int k = 0; k < K; ++k) {
                uint32_t m = active[k];
                const int c = __popc(m);
                if (r < c) {
                    for (int u = 0; u < r; ++u) m &= m - 1u;   // drop the r lowest decoding frames
                    s_pair[tid] = (uint8_t)(k << 5 | (__ffs(m) - 1));
                    break;
                }
                r -= c;
            }
        }
        __syncthreads();
    };
    // ---- stopping test of the tiles' current hard decisions: one lane per
    // (check, tile) covers all the tile's frames; frames failing a check are
    // OR-ed into the leader's word of their tile
    auto parity = [&]() {
        for (int k = 0; k < K; ++k) {
            uint32_t bad = 0;
            if (active[k])
                for (int c = gw * 32 + lane; c < M; c += TW * 32) {
                    const int32_t beg = __ldg(G.rp + c), d = __ldg(G.rp + c + 1) - beg;
                    bad |= plan_parity_word<8>(G.ci, beg, d, hdt[k], __ldcg(swt[k] + c));
                    pwords += d;
                }
            bad = __reduce_or_sync(0xffffffffu, bad & active[k]);
            if (lane == 0 && bad) atomicOr(unsat_dst + k, bad);
        }
    };
    // retire the frames whose test passed (iterations executed: t)
    auto retire = [&](int t) {
        plan_sync(tcs);
        for (int k = 0; k < K; ++k) {
            const uint32_t u = reinterpret_cast<volatile uint32_t *>(unsat_dst)[k];
            const uint32_t done = active[k] & ~u;
            if (trank == 0 && tid < nf[k] && ((done >> tid) & 1u)) G.iters[f0[k] + tid] = t;
            active[k] &= u;
        }
        plan_sync(tcs);   // every CTA has read the words before they are cleared
        if (trank == 0 && tid < K) s_unsat[tid] = 0;
        sparse_setup();
    };
    auto any_active = [&]() {
        uint32_t x = 0;
        for (int k = 0; k < K; ++k) x |= active[k];
        return x != 0;
    };
    sparse_setup();
    if (a.early_stop) {
        parity();
        retire(0);
    }
    for (int t = 1; t <= a.max_iter && any_active(); ++t) {
        const bool first = t == 1;
        for (int ly = 0; ly < G.n_layers; ++ly) {
            const int32_t lb = __ldg(G.lptr + ly), le = __ldg(G.lptr + ly + 1);
            if (sparse) {
                const int64_t ntask = (int64_t)(le - lb) * sA;
                for (int64_t t0 = (int64_t)gw * (32 / kSG); t0 < ntask; t0 += (int64_t)TW * (32 / kSG)) {
                    const int64_t t = t0 + stask;
                    const bool live = t < ntask;
                    const int32_t c = __ldg(G.lchk + lb + (live ? t / sA : 0));
                    const int pr = live ? s_pair[t % sA] : 0, pk = pr >> 5, pf = pr & 31;
                    const int32_t beg = __ldg(G.rp + c), d = __ldg(G.rp + c + 1) - beg;
                    const uint32_t neg0 = live ? (__ldcg(swt[pk] + c) >> pf) & 1u : 0u;
                    plan_check_task<SE>(G.ci, beg, d, first, Lt[pk] + pf, mt[pk] + pf, FT, neg0, live, sg, a.beta,
                                        hdt[pk], pf);
                    if (live && sg == 0) {
                        units += d;
                        if (first) units_first += d;
                    }
                }
            } else {
                for (int32_t kk = lb + gw * slots + slot; kk < le; kk += TW * slots) {
                    const int32_t c = __ldg(G.lchk + kk);
                    const int32_t beg = __ldg(G.rp + c), d = __ldg(G.rp + c + 1) - beg;
                    for (int k = 0; k < K; ++k) {
                        const uint32_t la = (active[k] >> f_lo) & vmask;   // this lane's frames still decoding
                        if (!la) continue;
                        plan_check<V, CH, SF>(G.ci, beg, d, first, Lt[k] + f_lo, mt[k] + f_lo, FT,
                                          (__ldcg(swt[k] + c) >> f_lo) & vmask, la, tr + lane * V, a.beta, hdt[k],
                                          f_lo);
                        const uint32_t na = (uint32_t)__popc(la);
                        units += d * na;
                        if (first) units_first += d * na;
                    }
                }
            }
            plan_sync(tcs);
        }
        if (a.early_stop || t == a.max_iter) {
            parity();
            retire(t);
        }
    }
    if (!a.early_stop && a.max_iter == 0) {
        parity();
        retire(0);
    }
    // ---- outputs: frames still active never satisfied the syndrome
    for (int k = 0; k < K; ++k) {
        if (trank == 0 && tid < nf[k]) {
            const bool act = (active[k] >> tid) & 1u;
            G.conv[f0[k] + tid] = act ? 0 : 1;
            if (act) G.iters[f0[k] + tid] = a.max_iter;
        }
        const float *L = Lt[k];
        for (int64_t v0 = (int64_t)gw * 32; v0 < n; v0 += (int64_t)TW * 32) {
            for (int i0 = 0; i0 < 32 * FT; i0 += 32 * 8) {
                float t[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int idx = i0 + u * 32 + lane, j = idx / FT, fi = idx - j * FT;
                    t[u] = (idx < 32 * FT && v0 + j < n) ? __ldcg(L + (v0 + j) * FT + fi) : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int idx = i0 + u * 32 + lane, j = idx / FT, fi = idx - j * FT;
                    if (idx < 32 * FT) tr[fi * 32 + (j ^ fi)] = t[u];
                }
            }
            __syncwarp();
            const int64_t v = v0 + lane;
            if (v < n)
                for (int i = 0; i < nf[k]; ++i)
                    G.bits[(int64_t)(f0[k] + i) * n + v] = tr[i * 32 + (lane ^ i)] < 0.0f ? 1 : 0;
            __syncwarp();
        }
    }
    cnt.units += units;
    cnt.units_first += units_first;
    cnt.pwords += pwords;
}

// Persistent loop: the team (the whole cluster, or the CTA when CS = 1) takes
// items from the queue until it is empty.
template <int CH, int NT, int V>
__global__ void __launch_bounds__(NT, 1)
plan_layered_kernel(PlanArgs a) {
    // [warps][SF][32] floats: q stash and 32 x 32 transposes
    extern __shared__ __align__(16) float qst[];
    __shared__ int s_item;
    __shared__ uint32_t s_unsat[kPlanMaxTiles];
    __shared__ uint8_t s_pair[kPlanMaxSparse];   // sparse mode: the item's decoding frames
    const int tid = threadIdx.x;
    const int CS = a.CS;
    const int rank = CS > 1 ? (int)cg::this_cluster().block_rank() : 0;
    volatile int *item_src = CS > 1 ? cg::this_cluster().map_shared_rank(&s_item, 0) : &s_item;
    uint32_t *unsat_dst = CS > 1 ? cg::this_cluster().map_shared_rank(s_unsat, 0) : s_unsat;
    PlanCount cnt;
    if (tid < kPlanMaxTiles) s_unsat[tid] = 0;
    for (;;) {
        if (rank == 0 && tid == 0) s_item = atomicAdd(a.head, 1);
        plan_sync(CS);
        const int item = *item_src;
        if (item >= a.n_items) {
            plan_sync(CS);   // no CTA leaves while another may still read the leader's word
            break;
        }
        plan_item<CH, V, (NT >= 512 ? 4 : 8), plan_stash_floats(NT)>(a, item, CS, rank, unsat_dst, s_unsat, qst, s_pair, cnt);
        plan_sync(CS);   // the tile is finished in every CTA before the leader takes the next
    }
    // per edge-frame update: posterior and message read and written (16 B; the
    // first iteration reads no message); per edge and tile of a stopping test:
    // the variable's hard-decision word gathered (4 B)
    prof_add(a.prof, cnt.units, cnt.units * 16 - cnt.units_first * 4 + cnt.pwords * 4);
}

}  // namespace qkd

// ------------------------------------------------------------------ host side
struct qkdrec_plan_s {
    std::vector<qkdrec_group> groups;
    qkdrec_decode_opts opts;
    qkdrec_tuning tuning;
    int32_t *d_head = nullptr;
    qkd::PlanGroup *d_groups = nullptr;
    qkd::PlanItem *d_items = nullptr;
    int32_t n_items = 0;
    size_t ws_needed = 0;      // for the current tuning
    size_t ws_max = 0;         // over every tuning the autotuner may pick
};

namespace qkd {

static const int kPlanFT[] = {8, 16, 32};
static const int kPlanThreads[] = {256, 512, 1024};
// load depth x threads per CTA: deeper chunks (fewer dependent round trips per
// check) need more registers, so they come with smaller CTAs
static const int kPlanDepth[] = {4, 8, 16};
// at two or four frames per lane every load holds V floats: depth 4 or 8 only,
// with half the threads of the one-frame variant of that depth
static int plan_max_threads(int depth, int V) {
    if (V == 1) return depth == 4 ? 1024 : (depth == 8 ? 512 : 256);
    return depth == 4 ? 512 : (depth == 8 ? 256 : 0);
}
static const int kPlanCS[] = {1, 2, 4, 8};
static const int kPlanTiles[] = {1, 2, 4};
static const int kPlanV[] = {1, 2, 4};
static const int kPlanSparse[] = {0, 1, 2, 4, 8};

template <size_t N>
static bool in_set(int v, const int (&set)[N]) {
    for (size_t i = 0; i < N; ++i)
        if (v == set[i]) return true;
    return false;
}

static bool tuning_ok(const qkdrec_tuning &t) {
    return in_set(t.frames_per_tile, kPlanFT) && in_set(t.threads_per_cta, kPlanThreads) &&
           in_set(t.stage_depth, kPlanDepth) && in_set(t.ctas_per_tile, kPlanCS) &&
           in_set(t.tiles_per_item, kPlanTiles) && in_set(t.frames_per_lane, kPlanV) &&
           t.frames_per_tile / t.frames_per_lane >= 8 && t.sparse_frames >= 0 && t.sparse_frames <= kPlanMaxSparse;
}

static size_t plan_ws_bytes(const std::vector<qkdrec_group> &gs, int FT) {
    size_t total = 0;
    for (const qkdrec_group &g : gs) {
        const CodeDev &d = g.code->d;
        total += (size_t)ceil_div(g.frames, FT) * (size_t)plan_tile_bytes(d.n, d.E, d.M, FT);
    }
    return total;
}

// (Re)build the device tables for the plan's current tuning (synchronous).
static qkdrec_status plan_build(qkdrec_plan_s &p) {
    const int FT = p.tuning.frames_per_tile;
    std::vector<PlanGroup> hg(p.groups.size());
    std::vector<PlanItem> items;
    std::vector<double> cost;
    int64_t off = 0;
    for (size_t i = 0; i < p.groups.size(); ++i) {
        const qkdrec_group &g = p.groups[i];
        const CodeDev &d = g.code->d;
        PlanGroup &G = hg[i];
        G.rp = d.rp;
        G.ci = d.ci;
        G.lptr = d.layer_ptr;
        G.lchk = d.layer_chk;
        G.llr = g.llr;
        G.synd = g.synd;
        G.bits = g.bits_out;
        G.iters = g.iters_out;
        G.conv = g.conv_out;
        G.ws_off = off;
        G.tile_bytes = plan_tile_bytes(d.n, d.E, d.M, FT);
        G.E = d.E;
        G.n = d.n;
        G.M = d.M;
        G.n_layers = d.n_layers;
        G.F = g.frames;
        G.dc_max = d.dc_max;
        const int tiles = (int)ceil_div(g.frames, FT);
        const int K = p.tuning.tiles_per_item;
        for (int t = 0; t < tiles; t += K) {
            const int nk = std::min(K, tiles - t);
            const double c = (double)d.E * (double)std::min(FT * nk, g.frames - t * FT);
            items.push_back(PlanItem{(int32_t)i, t, nk});
            cost.push_back(c + 1e-3 * (double)d.n_layers);
        }
        off += (int64_t)tiles * G.tile_bytes;
    }
    // longest first: the queue hands out the expensive tiles early
    std::vector<size_t> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<PlanItem> sorted(items.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
    cudaFree(p.d_groups);
    cudaFree(p.d_items);
    p.d_groups = nullptr;
    p.d_items = nullptr;
    QKD_CUDA(cudaMalloc(&p.d_groups, sizeof(PlanGroup) * std::max<size_t>(hg.size(), 1)));
    QKD_CUDA(cudaMalloc(&p.d_items, sizeof(PlanItem) * std::max<size_t>(sorted.size(), 1)));
    if (!hg.empty())
        QKD_CUDA(cudaMemcpy(p.d_groups, hg.data(), sizeof(PlanGroup) * hg.size(), cudaMemcpyHostToDevice));
    if (!sorted.empty())
        QKD_CUDA(cudaMemcpy(p.d_items, sorted.data(), sizeof(PlanItem) * sorted.size(), cudaMemcpyHostToDevice));
    p.n_items = (int32_t)sorted.size();
    p.ws_needed = (size_t)off;
    return QKDREC_OK;
}

template <int CH, int NT, int V>
static qkdrec_status plan_launch_ch(const PlanArgs &a, int threads, int CS, int n_items, cudaStream_t st) {
    // 128 KB of stash: above the default 48 KB of dynamic shared memory
    static bool attr_set = false;
    const size_t stash = (size_t)threads * plan_stash_floats(NT) * sizeof(float);
    if (!attr_set) {
        QKD_CUDA(cudaFuncSetAttribute(plan_layered_kernel<CH, NT, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((size_t)NT * plan_stash_floats(NT) * sizeof(float))));
        attr_set = true;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = stash;
    cfg.stream = st;
    int groups_resident = 0;
    if (CS > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(CS);
        QKD_CUDA(cudaOccupancyMaxActiveClusters(&groups_resident, plan_layered_kernel<CH, NT, V>, &cfg));
    } else {
        int per_sm = 0;
        QKD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_layered_kernel<CH, NT, V>, threads, stash));
        groups_resident = per_sm * sm_count();
    }
    if (groups_resident < 1)
        QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "launch shape %d threads x %d CTAs does not fit", threads, CS);
    const int groups = std::min(groups_resident, n_items);
    cfg.gridDim = dim3((unsigned)(groups * CS));
    QKD_CUDA(cudaLaunchKernelEx(&cfg, plan_layered_kernel<CH, NT, V>, a));
    return QKDREC_OK;
}

static qkdrec_status plan_launch(const qkdrec_plan_s &p, void *ws, size_t bytes, cudaStream_t st) {
    if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) QKD_FAIL(QKDREC_ERR_ARG, "workspace NULL or not 256-byte aligned");
    if (bytes < p.ws_needed) QKD_FAIL(QKDREC_ERR_ARG, "workspace %zu < %zu bytes", bytes, p.ws_needed);
    if (p.n_items == 0) return QKDREC_OK;
    PlanArgs a;
    a.groups = p.d_groups;
    a.items = p.d_items;
    a.n_items = p.n_items;
    a.head = p.d_head;
    a.ws = reinterpret_cast<char *>(ws);
    a.FT = p.tuning.frames_per_tile;
    a.CS = p.tuning.ctas_per_tile;
    a.max_iter = p.opts.max_iter;
    a.early_stop = p.opts.early_stop ? 1 : 0;
    a.sparse = p.tuning.sparse_frames;
    a.beta = p.opts.offset;
    a.prof = prof::counters(prof::kPlan);
    QKD_CUDA(cudaMemsetAsync(p.d_head, 0, sizeof(int32_t), st));
    const int threads = p.tuning.threads_per_cta;
    prof::Scope ps(prof::kPlan, st);
    const int dep = p.tuning.stage_depth, V = p.tuning.frames_per_lane;
    if (threads > plan_max_threads(dep, V))
        QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "load depth %d at %d frames per lane runs at most %d threads per CTA", dep, V,
                 plan_max_threads(dep, V));
    qkdrec_status s;
    if (V == 1)
        s = dep == 4   ? plan_launch_ch<4, 1024, 1>(a, threads, a.CS, p.n_items, st)
            : dep == 8 ? plan_launch_ch<8, 512, 1>(a, threads, a.CS, p.n_items, st)
                       : plan_launch_ch<16, 256, 1>(a, threads, a.CS, p.n_items, st);
    else if (V == 2)
        s = dep == 4 ? plan_launch_ch<4, 512, 2>(a, threads, a.CS, p.n_items, st)
                     : plan_launch_ch<8, 256, 2>(a, threads, a.CS, p.n_items, st);
    else
        s = dep == 4 ? plan_launch_ch<4, 512, 4>(a, threads, a.CS, p.n_items, st)
                     : plan_launch_ch<8, 256, 4>(a, threads, a.CS, p.n_items, st);
    if (s != QKDREC_OK) return s;
    QKD_LAUNCHED("plan_layered_kernel");
    return QKDREC_OK;
}

}  // namespace qkd

extern "C" {

void qkdrec_tuning_default(qkdrec_tuning *t) {
    if (!t) return;
    t->frames_per_tile = 32;
    t->threads_per_cta = 512;
    t->stage_depth = 8;
    t->ctas_per_tile = 4;
    t->tiles_per_item = 1;
    t->frames_per_lane = 1;
    t->sparse_frames = 4;
}

qkdrec_status qkdrec_plan_create(const qkdrec_group *groups, int32_t n_groups, const qkdrec_decode_opts *opts,
                                 const qkdrec_tuning *tuning, qkdrec_plan_t *out) {
    clear_error();
    if (!out) QKD_FAIL(QKDREC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_groups < 0 || (n_groups > 0 && !groups)) QKD_FAIL(QKDREC_ERR_ARG, "bad group list");
    if (!opts_ok(opts)) QKD_FAIL(QKDREC_ERR_ARG, "bad decode options");
    if (opts->algo != QKDREC_OMS_LAYERED || opts->prec != QKDREC_F32)
        QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "batched plans decode with FP32 layered offset min-sum");
    qkdrec_tuning tu;
    qkdrec_tuning_default(&tu);
    if (tuning) tu = *tuning;
    if (!tuning_ok(tu)) QKD_FAIL(QKDREC_ERR_ARG, "tuning outside the supported sets");
    for (int32_t i = 0; i < n_groups; ++i) {
        const qkdrec_group &g = groups[i];
        if (!g.code || g.frames < 0) QKD_FAIL(QKDREC_ERR_ARG, "group %d: NULL code or frames < 0", i);
        if (g.frames > 0 && (!g.llr || !g.synd || !g.bits_out || !g.iters_out || !g.conv_out))
            QKD_FAIL(QKDREC_ERR_ARG, "group %d: NULL input/output", i);
        // tile offsets are 32-bit: edges x 32 frames must stay below 2^32
        if ((uint64_t)g.code->d.E * 32u > 0xffffffffull)
            QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "group %d: %lld edges, above 2^27", i, (long long)g.code->d.E);
    }
    qkdrec_plan_s *p = new (std::nothrow) qkdrec_plan_s();
    if (!p) QKD_FAIL(QKDREC_ERR_NOMEM, "host allocation");
    p->groups.assign(groups, groups + n_groups);
    p->opts = *opts;
    p->tuning = tu;
    cudaError_t e = cudaMalloc(&p->d_head, sizeof(int32_t));
    if (e != cudaSuccess) {
        delete p;
        QKD_FAIL(QKDREC_ERR_NOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
    for (int ft : kPlanFT) p->ws_max = std::max(p->ws_max, plan_ws_bytes(p->groups, ft));
    qkdrec_status s = plan_build(*p);
    if (s != QKDREC_OK) {
        cudaFree(p->d_head);
        cudaFree(p->d_groups);
        cudaFree(p->d_items);
        delete p;
        return s;
    }
    *out = p;
    return QKDREC_OK;
}

void qkdrec_plan_destroy(qkdrec_plan_t p) {
    if (!p) return;
    cudaFree(p->d_head);
    cudaFree(p->d_groups);
    cudaFree(p->d_items);
    delete p;
}

qkdrec_status qkdrec_plan_workspace_size(qkdrec_plan_t p, size_t *bytes) {
    clear_error();
    if (!p || !bytes) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    *bytes = std::max<size_t>(p->ws_max, 256);
    return QKDREC_OK;
}

qkdrec_status qkdrec_plan_launch(qkdrec_plan_t p, void *workspace, size_t workspace_bytes, void *stream) {
    clear_error();
    if (!p) QKD_FAIL(QKDREC_ERR_ARG, "plan is NULL");
    return plan_launch(*p, workspace, workspace_bytes, as_stream(stream));
}

qkdrec_status qkdrec_plan_get_tuning(qkdrec_plan_t p, qkdrec_tuning *out) {
    clear_error();
    if (!p || !out) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    *out = p->tuning;
    return QKDREC_OK;
}

qkdrec_status qkdrec_plan_autotune(qkdrec_plan_t p, void *workspace, size_t workspace_bytes, int32_t max_iter,
                                   void *stream, qkdrec_tuning *best_out, float *best_ms) {
    clear_error();
    if (!p) QKD_FAIL(QKDREC_ERR_ARG, "plan is NULL");
    if (workspace_bytes < p->ws_max) QKD_FAIL(QKDREC_ERR_ARG, "workspace %zu < %zu bytes", workspace_bytes, p->ws_max);
    cudaStream_t st = as_stream(stream);
    const qkdrec_decode_opts keep = p->opts;
    if (max_iter > 0) p->opts.max_iter = std::min(max_iter, keep.max_iter);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    QKD_CUDA(cudaEventCreate(&e0));
    QKD_CUDA(cudaEventCreate(&e1));
    qkdrec_tuning best = p->tuning;
    float best_t = INFINITY;
    // time one shape: 1 = timed, 0 = does not fit on the device (skipped), < 0 = error
    auto trial = [&]() -> int {
        if (plan_launch(*p, workspace, workspace_bytes, st) != QKDREC_OK) {   // warm-up
            cudaGetLastError();
            clear_error();
            return 0;
        }
        cudaEventRecord(e0, st);
        if (plan_launch(*p, workspace, workspace_bytes, st) != QKDREC_OK) return -1;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_t) {
            best_t = ms;
            best = p->tuning;
        }
        return 1;
    };
    qkdrec_status s = QKDREC_OK;
    for (int ft : kPlanFT) {
        for (int nk : kPlanTiles) {
            p->tuning.frames_per_tile = ft;
            p->tuning.tiles_per_item = nk;
            if ((s = plan_build(*p)) != QKDREC_OK) break;
            for (int v : kPlanV)
                for (int cs : kPlanCS)
                    for (int th : kPlanThreads)
                        for (int dep : kPlanDepth) {
                            if (s != QKDREC_OK || ft / v < 8 || th > plan_max_threads(dep, v)) continue;
                            p->tuning.frames_per_lane = v;
                            p->tuning.ctas_per_tile = cs;
                            p->tuning.threads_per_cta = th;
                            p->tuning.stage_depth = dep;
                            if (trial() < 0) s = QKDREC_ERR_CUDA;
                        }
            if (s != QKDREC_OK) break;
        }
        if (s != QKDREC_OK) break;
    }
    // the sparse-mode threshold, at the fastest shape found
    if (s == QKDREC_OK && best_t < INFINITY) {
        p->tuning = best;
        if ((s = plan_build(*p)) == QKDREC_OK)
            for (int sp : kPlanSparse) {
                p->tuning.sparse_frames = sp;
                if (trial() < 0) {
                    s = QKDREC_ERR_CUDA;
                    break;
                }
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->opts = keep;
    p->tuning = best;
    qkdrec_status s2 = plan_build(*p);
    if (s != QKDREC_OK) return s;
    if (s2 != QKDREC_OK) return s2;
    QKD_CUDA(cudaStreamSynchronize(st));
    if (best_out) *best_out = best;
    if (best_ms) *best_ms = best_t;
    return QKDREC_OK;
}

}  // extern "C"

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
// leader's shared word), frames retiring one by one, the tile leaving early
// once all its frames are done.
//
// Lane layout: lane = slot * FT + frame, so a warp serves 32/FT checks at a
// time; with FT = 32 every posterior gather and message access of a warp is one
// 128-byte line.  Per tile the workspace holds L [n][FT] and m [E][FT] (frame
// fastest) and the tile's syndrome bits, one word per check.  Messages are not
// cleared: the first iteration reads m = 0 without loading it.  The q values of
// the first kStash edges of a check wait in shared memory between the two
// passes; the rest are recomputed from L and m, which no other check of the
// layer touches.  Posteriors go through L2 only (ld/st .cg), so what one SM of
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

struct PlanArgs {
    const PlanGroup *groups;
    const PlanItem *items;
    int32_t n_items;
    int32_t *head;
    char *ws;
    int32_t FT, CS, max_iter, early_stop;
    float beta;
    unsigned long long *prof;
};

static int64_t plan_tile_bytes(int64_t n, int64_t E, int64_t M, int FT) {
    return (int64_t)align_up((size_t)n * FT * 4, 256) + (int64_t)align_up((size_t)E * FT * 4, 256) +
           (int64_t)align_up((size_t)M * 4, 256);
}

// barrier over the CTAs that share a tile
__device__ __forceinline__ void plan_sync(int CS) {
    if (CS > 1) cg::this_cluster().sync();
    else __syncthreads();
}

// Per-launch work counters of one CTA.
struct PlanCount {
    unsigned long long units = 0, units_first = 0, punits = 0;
};

// Decode one work item -- K tiles of one group -- with a team of tcs CTAs
// (trank = this CTA's place in the team; unsat_dst = the team leader's shared
// stopping-test words, one per tile).  The K tiles run their layers in step:
// between two barriers every warp handles its checks of the layer for each
// tile in turn, so a layer with few checks still gives the team K times the
// work per barrier.  Each tile's arithmetic is that of a one-tile item.
template <int CH>
__device__ __forceinline__ void plan_item(const PlanArgs &a, int item, int tcs, int trank, uint32_t *unsat_dst,
                                          uint32_t *s_unsat, float *qst, PlanCount &cnt) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int FT = a.FT, slots = 32 / FT, slot = lane / FT, fl = lane - slot * FT;
    const int gw = trank * nwarps + warp, TW = tcs * nwarps;          // warp within the team
    const int64_t gt = (int64_t)trank * blockDim.x + tid, TT = (int64_t)tcs * blockDim.x;
    float *my = qst + (warp * kStash) * 32 + lane;
    float *tr = qst + (warp * kStash) * 32;                           // this warp's 32 x 32 tile
    uint32_t units = 0, units_first = 0, punits = 0;   // this item's share (added to cnt at the end)
    const PlanItem itm = a.items[item];
    const PlanGroup &G = a.groups[itm.g];
    const int n = G.n, M = G.M, K = itm.ntiles;
    int f0[kPlanMaxTiles], nf[kPlanMaxTiles];
    float *Lt[kPlanMaxTiles], *mt[kPlanMaxTiles];
    uint32_t *swt[kPlanMaxTiles], active[kPlanMaxTiles];   // active: same value in every thread
#pragma unroll
    for (int k = 0; k < kPlanMaxTiles; ++k) {
        const int tile = itm.tile + min(k, K - 1);
        f0[k] = tile * FT;
        nf[k] = k < K ? min(FT, G.F - f0[k]) : 0;
        char *tb = a.ws + G.ws_off + (int64_t)tile * G.tile_bytes;
        Lt[k] = reinterpret_cast<float *>(tb);
        mt[k] = reinterpret_cast<float *>(tb + align_up((size_t)n * FT * 4, 256));
        swt[k] = reinterpret_cast<uint32_t *>(tb + align_up((size_t)n * FT * 4, 256) + align_up((size_t)G.E * FT * 4, 256));
        active[k] = nf[k] == 32 ? 0xffffffffu : ((1u << nf[k]) - 1u);
    }
    // ---- load the tiles: L[v][i] = llr[f0 + i][v] through a per-warp transpose
    // (swizzled columns, conflict-free), padding frames get a confident 0
    for (int k = 0; k < K; ++k) {
        float *L = Lt[k];
        for (int64_t v0 = (int64_t)gw * 32; v0 < n; v0 += (int64_t)TW * 32) {
            const int64_t v = v0 + lane;
            for (int i = 0; i < FT; ++i)
                tr[i * 32 + (lane ^ i)] = (i < nf[k] && v < n) ? __ldg(G.llr + (int64_t)(f0[k] + i) * n + v) : kLlrClip;
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
    // ---- stopping test of the tiles' current posteriors: frames failing a
    // check are OR-ed into the leader's word of their tile
    auto parity = [&]() {
        for (int k = 0; k < K; ++k) {
            uint32_t bad = 0;
            if (fl < nf[k] && ((active[k] >> fl) & 1u)) {
                const float *L = Lt[k];
                for (int c = gw * slots + slot; c < M; c += TW * slots) {
                    uint32_t par = (__ldcg(swt[k] + c) >> fl) & 1u;
                    const int32_t beg = __ldg(G.rp + c), d = __ldg(G.rp + c + 1) - beg;
                    // CH gathers in flight (indices past the last edge clamped to it)
                    for (int k0 = 0; k0 < d; k0 += CH) {
                        float Lv[CH];
#pragma unroll
                        for (int j = 0; j < CH; ++j)
                            Lv[j] = __ldcg(L + ((uint32_t)__ldg(G.ci + beg + min(k0 + j, d - 1)) * FT + fl));
#pragma unroll
                        for (int j = 0; j < CH; ++j)
                            if (k0 + j < d) par ^= (uint32_t)(Lv[j] < 0.0f);
                    }
                    bad |= par << fl;
                    punits += d;
                }
            }
            bad = __reduce_or_sync(0xffffffffu, bad);
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
    };
    auto any_active = [&]() {
        uint32_t x = 0;
        for (int k = 0; k < K; ++k) x |= active[k];
        return x != 0;
    };
    if (a.early_stop) {
        parity();
        retire(0);
    }
    for (int t = 1; t <= a.max_iter && any_active(); ++t) {
        const bool first = t == 1;
        for (int ly = 0; ly < G.n_layers; ++ly) {
            const int32_t lb = __ldg(G.lptr + ly), le = __ldg(G.lptr + ly + 1);
            for (int32_t kk = lb + gw * slots + slot; kk < le; kk += TW * slots) {
                const int32_t c = __ldg(G.lchk + kk);
                const int32_t beg = __ldg(G.rp + c), d = __ldg(G.rp + c + 1) - beg;
                for (int k = 0; k < K; ++k) {
                    if (!(fl < nf[k] && ((active[k] >> fl) & 1u))) continue;
                    float *L = Lt[k], *msg = mt[k];
                    uint32_t neg = (__ldcg(swt[k] + c) >> fl) & 1u;
                    float mn1 = INFINITY, mn2 = INFINITY;
                    int32_t arg = -1;
                    units += d;
                    if (first) units_first += d;
                    // pass 1: q = L - m on every edge (CH loads in flight, indices clamped)
                    for (int k0 = 0; k0 < d; k0 += CH) {
                        float Lv[CH], mo[CH];
#pragma unroll
                        for (int j = 0; j < CH; ++j) {
                            const int32_t e = beg + min(k0 + j, d - 1);
                            Lv[j] = __ldcg(L + ((uint32_t)__ldg(G.ci + e) * FT + fl));
                            mo[j] = first ? 0.0f : __ldcs(msg + ((uint32_t)e * FT + fl));
                        }
#pragma unroll
                        for (int j = 0; j < CH; ++j) {
                            const int kq = k0 + j;
                            if (kq >= d) break;
                            const float q = Lv[j] - mo[j];
                            if (kq < kStash) my[kq * 32] = q;
                            neg ^= (uint32_t)(q < 0.0f);
                            const float m = fabsf(q);
                            if (m < mn1) { mn2 = mn1; mn1 = m; arg = kq; }
                            else if (m < mn2) mn2 = m;
                        }
                    }
                    // pass 2: new messages and posteriors L = q + m
                    for (int kq = 0; kq < d; ++kq) {
                        const int32_t e = beg + kq;
                        float *Lp = L + ((uint32_t)__ldg(G.ci + e) * FT + fl);
                        float *mp = msg + ((uint32_t)e * FT + fl);
                        // edges beyond the stash: L and m of this edge are still unchanged
                        const float q = kq < kStash ? my[kq * 32] : __ldcg(Lp) - (first ? 0.0f : __ldcs(mp));
                        const float mag = fmaxf(((kq == arg) ? mn2 : mn1) - a.beta, 0.0f);
                        const float mn = ((neg ^ (uint32_t)(q < 0.0f)) & 1u) ? -mag : mag;
                        __stcs(mp, mn);
                        __stcg(Lp, q + mn);
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
            for (int idx = lane; idx < 32 * FT; idx += 32) {
                const int j = idx / FT, fi = idx - j * FT;
                tr[fi * 32 + (j ^ fi)] = v0 + j < n ? __ldcg(L + (v0 + j) * FT + fi) : 0.0f;
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
    cnt.punits += punits;
}

// Persistent loop: the team (the whole cluster, or the CTA when CS = 1) takes
// items from the queue until it is empty.
template <int CH, int NT>
__global__ void __launch_bounds__(NT, 1)
plan_layered_kernel(PlanArgs a) {
    extern __shared__ float qst[];  // [warps][kStash][32]: q stash; 32 x 32 transposes
    __shared__ int s_item;
    __shared__ uint32_t s_unsat[kPlanMaxTiles];
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
        plan_item<CH>(a, item, CS, rank, unsat_dst, s_unsat, qst, cnt);
        plan_sync(CS);   // the tile is finished in every CTA before the leader takes the next
    }
    // per edge-frame update: posterior and message read and written (16 B; the
    // first iteration reads no message); per edge-frame of a stopping test: the
    // posterior gathered (4 B)
    prof_add(a.prof, cnt.units, cnt.units * 16 - cnt.units_first * 4 + cnt.punits * 4);
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
static int plan_max_threads(int depth) { return depth == 4 ? 1024 : (depth == 8 ? 512 : 256); }
static const int kPlanCS[] = {1, 2, 4, 8};
static const int kPlanTiles[] = {1, 2, 4};

template <size_t N>
static bool in_set(int v, const int (&set)[N]) {
    for (size_t i = 0; i < N; ++i)
        if (v == set[i]) return true;
    return false;
}

static bool tuning_ok(const qkdrec_tuning &t) {
    return in_set(t.frames_per_tile, kPlanFT) && in_set(t.threads_per_cta, kPlanThreads) &&
           in_set(t.stage_depth, kPlanDepth) && in_set(t.ctas_per_tile, kPlanCS) &&
           in_set(t.tiles_per_item, kPlanTiles);
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

template <int CH, int NT>
static qkdrec_status plan_launch_ch(const PlanArgs &a, int threads, int CS, int n_items, cudaStream_t st) {
    // up to 1024 threads x 128 B of stash: above the default 48 KB of dynamic shared memory
    static bool attr_set = false;
    const size_t stash = (size_t)(threads / 32) * kStash * 32 * sizeof(float);
    if (!attr_set) {
        QKD_CUDA(cudaFuncSetAttribute(plan_layered_kernel<CH, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)((size_t)(NT / 32) * kStash * 32 * sizeof(float))));
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
        QKD_CUDA(cudaOccupancyMaxActiveClusters(&groups_resident, plan_layered_kernel<CH, NT>, &cfg));
    } else {
        int per_sm = 0;
        QKD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, plan_layered_kernel<CH, NT>, threads, stash));
        groups_resident = per_sm * sm_count();
    }
    if (groups_resident < 1)
        QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "launch shape %d threads x %d CTAs does not fit", threads, CS);
    const int groups = std::min(groups_resident, n_items);
    cfg.gridDim = dim3((unsigned)(groups * CS));
    QKD_CUDA(cudaLaunchKernelEx(&cfg, plan_layered_kernel<CH, NT>, a));
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
    a.beta = p.opts.offset;
    a.prof = prof::counters(prof::kPlan);
    QKD_CUDA(cudaMemsetAsync(p.d_head, 0, sizeof(int32_t), st));
    const int threads = p.tuning.threads_per_cta;
    prof::Scope ps(prof::kPlan, st);
    if (threads > plan_max_threads(p.tuning.stage_depth))
        QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "load depth %d runs at most %d threads per CTA", p.tuning.stage_depth,
                 plan_max_threads(p.tuning.stage_depth));
    qkdrec_status s = p.tuning.stage_depth == 4   ? plan_launch_ch<4, 1024>(a, threads, a.CS, p.n_items, st)
                      : p.tuning.stage_depth == 8 ? plan_launch_ch<8, 512>(a, threads, a.CS, p.n_items, st)
                                                  : plan_launch_ch<16, 256>(a, threads, a.CS, p.n_items, st);
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
            for (int cs : kPlanCS)
                for (int th : kPlanThreads)
                    for (int dep : kPlanDepth) {
                        if (s != QKDREC_OK) continue;
                        p->tuning.ctas_per_tile = cs;
                        p->tuning.threads_per_cta = th;
                        p->tuning.stage_depth = dep;
                        if (trial() < 0) s = QKDREC_ERR_CUDA;
                    }
            if (s != QKDREC_OK) break;
        }
        if (s != QKDREC_OK) break;
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

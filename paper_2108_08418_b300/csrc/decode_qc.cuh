// Layered offset min-sum for quasi-cyclic codes with TMA staging (included by
// decode.cu inside namespace qkd, after decode_layered.cuh).
//
// Layer i of a quasi-cyclic code is base row i: check z of the layer touches,
// through base column k, variable k Z + (z + s_ik) mod Z.  So the checks
// z0 .. z0+Zc-1 of a layer touch, per base column, the contiguous (cyclic) run
// of Zc variables starting at (z0 + s_ik) mod Z -- for one 32-frame block that
// is a Zc x 128-byte tile of the posterior array, which one TMA tile copy
// brings into shared memory (two copies where the run wraps around the
// circulant; the out-of-range rows of each copy read as zero and are not
// used).  A CTA takes one chunk of Zc checks of the layer for one frame block
// (grid-stride over the list of frame blocks still decoding), waits for its
// copies on an mbarrier (bounded: after kQcMaxSpins polls it records a timeout
// and leaves the chunk undecoded), then runs the same check update as the
// generic layered kernel -- q = L - m in edge order, min / second min / sign,
// m = (-1)^s prod sgn max(min - beta, 0), L = q + m -- with q kept in the tile.
// Messages are read and written with plain coalesced accesses (the edges of a
// check are consecutive), posteriors written back with plain stores (a TMA
// store cannot start at the negative row of a wrapped run).  Every variable
// lies in exactly one check per base row, so the CTAs of one layer never touch
// the same posterior.

constexpr uint32_t kQcMaxSpins = 1u << 24;

struct QcLayer {
    const int32_t *shift;   // [mb][nb]
    int32_t Z, nb, row, Zc;
    int32_t *timeouts;      // incremented when a CTA gives up waiting for its copies
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 4-D tile copy global -> shared completing on `bar` (coordinates innermost first)
__device__ __forceinline__ void tma_load_4d(float *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];"
        :
        : "r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w),
          "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(float *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];"
        :
        : "r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// 3-D tile copy shared -> global (bulk group of the issuing thread)
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int x, int y, int z, const float *src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];"
                 :
                 : "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(src))
                 : "memory");
}

__global__ void __launch_bounds__(256)
layer_qc_tma(DecArgs a, const __grid_constant__ CUtensorMap tmL, const __grid_constant__ CUtensorMap tmM,
             QcLayer q) {
    extern __shared__ __align__(128) float smem_raw[];
    __shared__ __align__(8) uint64_t bar[2];
    const int Z = q.Z, nb = q.nb, Zc = q.Zc, row = q.row;
    // two stages of posterior tiles [nb][2][Zc][32] and a message tile
    // [Zc nb][32] (the edges of the chunk's checks are consecutive), 128-byte
    // aligned for the tile copies (128 spare bytes allocated): the copies for
    // the next frame block are in flight while this one is decoded
    float *stage0 = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    const size_t stage_floats = (size_t)3 * nb * Zc * 32;
    const int z0 = blockIdx.x * Zc;
    const int zn = min(Zc, Z - z0);           // checks of this chunk
    const int64_t e_first = ((int64_t)row * Z + z0) * nb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    float *L = reinterpret_cast<float *>(a.L);
    float *msg = reinterpret_cast<float *>(a.msg);
    const int32_t *sh = q.shift + row * nb;
    const uint32_t tile_bytes = (uint32_t)Zc * 32u * 4u;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // thread 0: the tile copies of frame block fb into stage st
    auto issue = [&](int32_t fb, int st) {
        float *tiles = stage0 + st * stage_floats;
        uint32_t bytes = (uint32_t)nb * tile_bytes;   // the message tile
        for (int k = 0; k < nb; ++k) {
            const int y0 = (z0 + __ldg(sh + k)) % Z;
            bytes += (y0 + Zc > Z ? 2u : 1u) * tile_bytes;
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&bar[st])), "r"(bytes)
                     : "memory");
        for (int k = 0; k < nb; ++k) {
            const int y0 = (z0 + __ldg(sh + k)) % Z;
            tma_load_4d(tiles + (size_t)(2 * k) * Zc * 32, &tmL, 0, y0, k, fb, &bar[st]);
            if (y0 + Zc > Z) tma_load_4d(tiles + (size_t)(2 * k + 1) * Zc * 32, &tmL, 0, y0 - Z, k, fb, &bar[st]);
        }
        // messages of the chunk's edges (rows past the last edge read as zero)
        tma_load_3d(tiles + (size_t)2 * nb * Zc * 32, &tmM, 0, (int)e_first, fb, &bar[st]);
    };
    uint32_t phase[2] = {0u, 0u};
    unsigned long long units = 0;
    const int32_t nblk = *a.blk_n;
    if (threadIdx.x == 0 && (int32_t)blockIdx.y < nblk) issue(__ldg(a.blk + blockIdx.y), 0);
    int it = 0;
    for (int32_t bi = blockIdx.y; bi < nblk; bi += gridDim.y, ++it) {
        const int cur = it & 1;
        const int32_t fb = __ldg(a.blk + bi);
        // the other stage was released by the barrier that ended the previous block,
        // and its message tile has been read out by the store of that block
        if (threadIdx.x == 0 && bi + (int32_t)gridDim.y < nblk) {
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            issue(__ldg(a.blk + bi + gridDim.y), cur ^ 1);
        }
        bool ok = false;
        for (uint32_t spins = 0; spins < kQcMaxSpins; ++spins)
            if (mbar_try_wait(&bar[cur], phase[cur])) {
                ok = true;
                break;
            }
        phase[cur] ^= 1u;
        if (!__syncthreads_and(ok)) {
            // the copies did not arrive: record it, give copies still in flight
            // (both stages) a second bounded wait before the shared memory is
            // released, and leave the remaining blocks undecoded
            if (threadIdx.x == 0) {
                atomicAdd(q.timeouts, 1);
                asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                for (uint32_t spins = 0; spins < kQcMaxSpins && !mbar_try_wait(&bar[cur], phase[cur] ^ 1u); ++spins) {
                }
                if (bi + (int32_t)gridDim.y < nblk)
                    for (uint32_t spins = 0; spins < kQcMaxSpins && !mbar_try_wait(&bar[cur ^ 1], phase[cur ^ 1]);
                         ++spins) {
                    }
            }
            __syncthreads();
            return;
        }
        float *tiles = stage0 + cur * stage_floats;
        float *mtile = tiles + (size_t)2 * nb * Zc * 32;
        const int64_t f = ((int64_t)fb << 5) + lane;
        const bool act = a.active[f] != 0;
        const int64_t bL = fpos(0, a.n, f, 5), bM = fpos(0, a.E, f, 5);
        for (int zz = warp; zz < Zc && z0 + zz < Z; zz += nwarps) {
            if (!act) continue;
            const int z = z0 + zz;
            const int32_t c = row * Z + z;
            uint32_t neg = (__ldg(a.sbits + (int64_t)c * a.W + (f >> 5)) >> (f & 31)) & 1u;
            float mn1 = INFINITY, mn2 = INFINITY;
            int arg = -1;
            units += nb;
            // pass 1: q = L - m, kept in the tile slot of this lane
            for (int k = 0; k < nb; ++k) {
                const int y0 = (z0 + __ldg(sh + k)) % Z;
                float *slot = tiles + ((size_t)(2 * k + (y0 + zz < Z ? 0 : 1)) * Zc + zz) * 32 + lane;
                const float qv = *slot - mtile[((size_t)zz * nb + k) * 32 + lane];
                *slot = qv;
                neg ^= (uint32_t)(qv < 0.0f);
                const float mq = fabsf(qv);
                if (mq < mn1) { mn2 = mn1; mn1 = mq; arg = k; }
                else if (mq < mn2) mn2 = mq;
            }
            // pass 2: new messages and posteriors
            for (int k = 0; k < nb; ++k) {
                const int s = __ldg(sh + k);
                const int y0 = (z0 + s) % Z;
                const float qv = tiles[((size_t)(2 * k + (y0 + zz < Z ? 0 : 1)) * Zc + zz) * 32 + lane];
                const float mag = fmaxf(((k == arg) ? mn2 : mn1) - a.beta, 0.0f);
                const float mv = ((neg ^ (uint32_t)(qv < 0.0f)) & 1u) ? -mag : mag;
                mtile[((size_t)zz * nb + k) * 32 + lane] = mv;
                L[bL + ((int64_t)(k * Z + (z + s) % Z) << 5)] = qv + mv;
            }
        }
        // retired frames keep their messages: the tile still holds the loaded
        // values.  The tile's shared-memory writes are made visible to the copy
        // engine, then one tile copy stores the chunk's messages.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            if (zn == Zc) tma_store_3d(&tmM, 0, (int)e_first, fb, mtile);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
        if (zn < Zc) {
            // a short last chunk: its rows end before the tile does, store them plainly
            for (int r = warp; r < zn * nb; r += nwarps) msg[bM + ((e_first + r) << 5)] = mtile[(size_t)r * 32 + lane];
        }
        __syncthreads();   // this stage is refilled two blocks later
    }
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    // posterior and message read and written per updated edge-frame
    prof_add(a.prof, units, units * 16);
}

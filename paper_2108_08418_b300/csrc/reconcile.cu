// qkdrec_reconcile: one block of quadrature pairs through the whole reverse
// slice reconciliation (Sec. II Steps 4-5, Sec. III-A/B): Bob's quantiser and
// slices, his syndromes, then per slice Alice's soft information from x and her
// already reconciled lower slices and the BP decode of every sub-block; the
// reconciled slices leave packed eight bits to a byte.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "profile.cuh"

namespace qkd {

__global__ void pack_frames_kernel(const uint8_t *__restrict__ bits, int32_t n, int32_t F, int64_t Wt,
                                   uint32_t *__restrict__ bitsT);
__global__ void syndrome_packed_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                       const uint32_t *__restrict__ bitsT, int32_t n, int32_t M, int64_t Wt,
                                       int64_t W, uint32_t *__restrict__ sbits, unsigned long long *prof);

// Memory a pointer refers to, for the host-or-device arguments.
static bool device_reachable(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // plain host memory on some drivers: clear the sticky-free error
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Workspace: a shared part (host x, y staging; Bob's slices and their packed
// staging) and one slot per partition in flight (Alice's slices, one LLR
// plane, Bob's packed frames and syndromes, the decoder workspace, staging of
// the host outputs).  Partitions are independent, so with k slots k of them
// decode at once on side streams; a slot is reused by the partitions of its
// stream in order.
struct RecLayout {
    size_t xs, ys, bob, bpk, shared;              // shared part
    size_t alice, llr, bitsT, sbits, dec, pk, cv, it, slot;   // offsets inside a slot; slot size
    size_t dec_bytes;
    int32_t fmax;
};

static qkdrec_status rec_layout(int64_t count, int32_t m, const qkdrec_decode_opts *opts, const qkdrec_point *pts,
                                int32_t np, RecLayout &l) {
    size_t bitsT = 0, sbits = 0, dec = 0;
    int32_t fmax = 0;
    for (int32_t p = 0; p < np; ++p) {
        const int32_t n = pts[p].n;
        const int64_t F = count / n, W = ceil_div(F, 32);
        fmax = std::max<int32_t>(fmax, (int32_t)F);
        bitsT = std::max<size_t>(bitsT, (size_t)W * n * 4);
        for (int32_t j = 0; j < m; ++j) {
            const qkdrec_code_t c = pts[p].codes[j];
            if (!c) continue;
            size_t b = 0;
            qkdrec_status s = qkdrec_decode_workspace_size(c, (int32_t)F, opts, &b);
            if (s != QKDREC_OK) return s;
            dec = std::max(dec, b);
            sbits = std::max<size_t>(sbits, (size_t)c->d.M * W * 4);
        }
    }
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + std::max<size_t>(bytes, 1), 256); return o; };
    l.xs = take((size_t)count * 4);
    l.ys = take((size_t)count * 4);
    l.bob = take((size_t)m * count);
    l.bpk = take((size_t)m * count / 8);
    l.shared = off;
    off = 0;
    l.alice = take((size_t)m * count);
    l.llr = take((size_t)count * 4);
    l.bitsT = take(bitsT);
    l.sbits = take(sbits);
    l.dec = take(dec);
    l.dec_bytes = dec;
    l.pk = take((size_t)m * count / 8);
    l.cv = take((size_t)m * fmax);
    l.it = take((size_t)m * fmax * 4);
    l.slot = off;
    l.fmax = fmax;
    return QKDREC_OK;
}

// Side streams and events of this device for partitions in flight, created at
// the first call that runs more than one (outside stream capture) and kept.
constexpr int kRecSlots = 8;
struct SidePool {
    bool ok = false;
    cudaStream_t st[kRecSlots];
    cudaEvent_t fork, join[kRecSlots];
};
static std::mutex g_pool_mu;
static SidePool g_pool[64];

static qkdrec_status side_pool(SidePool **out) {
    int dev = 0;
    QKD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "device index %d above 63", dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    SidePool &sp = g_pool[dev];
    if (!sp.ok) {
        // all or nothing: a failed creation releases what was made
        SidePool np;
        int ns = 0, ne = 0;
        bool fork = false;
        cudaError_t e = cudaEventCreateWithFlags(&np.fork, cudaEventDisableTiming);
        fork = e == cudaSuccess;
        for (int k = 0; k < kRecSlots && e == cudaSuccess; ++k) {
            if ((e = cudaStreamCreateWithFlags(&np.st[k], cudaStreamNonBlocking)) != cudaSuccess) break;
            ++ns;
            if ((e = cudaEventCreateWithFlags(&np.join[k], cudaEventDisableTiming)) != cudaSuccess) break;
            ++ne;
        }
        if (e != cudaSuccess) {
            for (int k = 0; k < ns; ++k) cudaStreamDestroy(np.st[k]);
            for (int k = 0; k < ne; ++k) cudaEventDestroy(np.join[k]);
            if (fork) cudaEventDestroy(np.fork);
            QKD_FAIL(QKDREC_ERR_CUDA, "side streams for concurrent partitions: %s", cudaGetErrorString(e));
        }
        np.ok = true;
        sp = np;
    }
    *out = &sp;
    return QKDREC_OK;
}

static qkdrec_status rec_check(int64_t count, int32_t m, const qkdrec_decode_opts *opts, const qkdrec_point *pts,
                               int32_t np) {
    if (count <= 0 || count % 32) QKD_FAIL(QKDREC_ERR_ARG, "count=%lld must be a positive multiple of 32",
                                           (long long)count);
    if (m < 1 || m > 8) QKD_FAIL(QKDREC_ERR_ARG, "m_slices=%d outside [1, 8]", m);
    if (!opts) QKD_FAIL(QKDREC_ERR_ARG, "opts is NULL");
    if (np < 1 || !pts) QKD_FAIL(QKDREC_ERR_ARG, "need at least one sub-block length");
    for (int32_t p = 0; p < np; ++p) {
        const int32_t n = pts[p].n;
        if (n <= 0 || n % 32 || count % n)
            QKD_FAIL(QKDREC_ERR_ARG, "point %d: n=%d must be a positive multiple of 32 dividing count", p, n);
        if (count / n > (int64_t)65535 * 32) QKD_FAIL(QKDREC_ERR_ARG, "point %d: too many frames", p);
        if (!pts[p].codes || !pts[p].alice_packed) QKD_FAIL(QKDREC_ERR_ARG, "point %d: codes/alice_packed NULL", p);
        for (int32_t j = 0; j < m; ++j) {
            const qkdrec_code_t c = pts[p].codes[j];
            if (c && c->d.n != n) QKD_FAIL(QKDREC_ERR_ARG, "point %d slice %d: code length %d != n=%d", p, j, c->d.n, n);
        }
    }
    return QKDREC_OK;
}

// status of an enqueued runtime call
static qkdrec_status enq(cudaError_t e) {
    if (e == cudaSuccess) return QKDREC_OK;
    QKD_FAIL(QKDREC_ERR_CUDA, "%s", cudaGetErrorString(e));
}

// dst (host or device) <- src (device, in the workspace), on the stream
static qkdrec_status put(void *dst, const void *src, size_t bytes, cudaStream_t st) {
    if (!dst || !bytes) return QKDREC_OK;
    QKD_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    return QKDREC_OK;
}

}  // namespace qkd

using namespace qkd;

extern "C" {

qkdrec_status qkdrec_reconcile_workspace_size_limited(int64_t count, int32_t m_slices, const qkdrec_decode_opts *opts,
                                                      const qkdrec_point *points, int32_t n_points,
                                                      int32_t max_in_flight, size_t *bytes) {
    clear_error();
    if (!bytes) QKD_FAIL(QKDREC_ERR_ARG, "bytes is NULL");
    if (max_in_flight < 1) QKD_FAIL(QKDREC_ERR_ARG, "max_in_flight=%d must be >= 1", max_in_flight);
    qkdrec_status s = rec_check(count, m_slices, opts, points, n_points);
    if (s != QKDREC_OK) return s;
    RecLayout l;
    if ((s = rec_layout(count, m_slices, opts, points, n_points, l)) != QKDREC_OK) return s;
    const int32_t k = std::min(std::min(n_points, max_in_flight), (int32_t)kRecSlots);
    *bytes = l.shared + (size_t)k * l.slot;
    return QKDREC_OK;
}

qkdrec_status qkdrec_reconcile_workspace_size(int64_t count, int32_t m_slices, const qkdrec_decode_opts *opts,
                                              const qkdrec_point *points, int32_t n_points, size_t *bytes) {
    return qkdrec_reconcile_workspace_size_limited(count, m_slices, opts, points, n_points, kRecSlots, bytes);
}

qkdrec_status qkdrec_reconcile(const float *x, const float *y, int64_t count, int32_t m, double lo, double hi,
                               double sigma_n, qkdrec_label label, const qkdrec_decode_opts *opts,
                               const qkdrec_point *points, int32_t n_points, uint8_t *bob_packed, void *workspace,
                               size_t workspace_bytes, void *stream) {
    clear_error();
    qkdrec_status s = rec_check(count, m, opts, points, n_points);
    if (s != QKDREC_OK) return s;
    if (!x || !y) QKD_FAIL(QKDREC_ERR_ARG, "x/y NULL");
    if (!(lo < hi) || !(sigma_n > 0)) QKD_FAIL(QKDREC_ERR_ARG, "need lo < hi and sigma_n > 0");
    if (!workspace || reinterpret_cast<uintptr_t>(workspace) % 256)
        QKD_FAIL(QKDREC_ERR_ARG, "workspace NULL or not 256-byte aligned");
    RecLayout l;
    if ((s = rec_layout(count, m, opts, points, n_points, l)) != QKDREC_OK) return s;
    if (workspace_bytes < l.shared + l.slot)
        QKD_FAIL(QKDREC_ERR_ARG, "workspace %zu bytes < %zu needed", workspace_bytes, l.shared + l.slot);
    // partitions in flight: as many slots as the workspace holds
    const int32_t nslot = (int32_t)std::min<size_t>(
        std::min<size_t>((size_t)n_points, (size_t)kRecSlots), (workspace_bytes - l.shared) / l.slot);
    SidePool *pool = nullptr;
    if (nslot > 1 && (s = side_pool(&pool)) != QKDREC_OK) return s;
    cudaStream_t st = as_stream(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    // inputs: device memory is read in place, host memory copied in on the stream
    const float *xd = x, *yd = y;
    if (!device_reachable(x)) {
        QKD_CUDA(cudaMemcpyAsync(ws + l.xs, x, (size_t)count * 4, cudaMemcpyHostToDevice, st));
        xd = reinterpret_cast<const float *>(ws + l.xs);
    }
    if (!device_reachable(y)) {
        QKD_CUDA(cudaMemcpyAsync(ws + l.ys, y, (size_t)count * 4, cudaMemcpyHostToDevice, st));
        yd = reinterpret_cast<const float *>(ws + l.ys);
    }
    uint8_t *bob = reinterpret_cast<uint8_t *>(ws + l.bob);
    // Bob: quantiser and bit slices (Sec. III-B steps 1-2)
    if ((s = qkdrec_quantise_slices(yd, count, m, lo, hi, label, nullptr, bob, stream)) != QKDREC_OK) return s;
    const int64_t plane8 = count / 8;
    if (bob_packed) {
        const bool dev = device_reachable(bob_packed);
        uint8_t *bpk = reinterpret_cast<uint8_t *>(ws + l.bpk);
        for (int32_t j = 0; j < m; ++j)
            if ((s = qkdrec_pack_bits(bob + (size_t)j * count, count, dev ? bob_packed + j * plane8 : bpk + j * plane8,
                                      stream)) != QKDREC_OK)
                return s;
        if (!dev && (s = put(bob_packed, bpk, (size_t)m * plane8, st)) != QKDREC_OK) return s;
    }
    // fork: partition p runs on side stream p mod nslot, after Bob's slices
    if (pool) {
        QKD_CUDA(cudaEventRecord(pool->fork, st));
        for (int32_t k = 0; k < nslot; ++k) QKD_CUDA(cudaStreamWaitEvent(pool->st[k], pool->fork, 0));
    }
    for (int32_t p = 0; p < n_points && s == QKDREC_OK; ++p) {
        const qkdrec_point &pt = points[p];
        const int32_t n = pt.n, F = (int32_t)(count / n);
        const int64_t W = ceil_div(F, 32);
        cudaStream_t sp = pool ? pool->st[p % nslot] : st;
        void *spv = reinterpret_cast<void *>(sp);
        char *slot = ws + l.shared + (size_t)(p % nslot) * l.slot;
        uint8_t *alice = reinterpret_cast<uint8_t *>(slot + l.alice);
        float *llr = reinterpret_cast<float *>(slot + l.llr);
        uint32_t *bitsT = reinterpret_cast<uint32_t *>(slot + l.bitsT), *sbits = reinterpret_cast<uint32_t *>(slot + l.sbits);
        uint8_t *pk = reinterpret_cast<uint8_t *>(slot + l.pk), *cv = reinterpret_cast<uint8_t *>(slot + l.cv);
        int32_t *it = reinterpret_cast<int32_t *>(slot + l.it);
        const bool dev_a = device_reachable(pt.alice_packed);
        const bool dev_c = !pt.converged || device_reachable(pt.converged);
        const bool dev_i = !pt.iters || device_reachable(pt.iters);
        uint8_t *cv_out = pt.converged && dev_c ? pt.converged : cv;
        int32_t *it_out = pt.iters && dev_i ? pt.iters : it;
        for (int32_t j = 0; j < m; ++j) {
            const qkdrec_code_t c = pt.codes[j];
            uint8_t *aj = alice + (size_t)j * count;
            if (!c) {
                // disclosed slice (rate 0): Bob's bits are sent in the clear
                if ((s = enq(cudaMemcpyAsync(aj, bob + (size_t)j * count, (size_t)count, cudaMemcpyDeviceToDevice,
                                             sp))) != QKDREC_OK ||
                    (s = enq(cudaMemsetAsync(cv_out + (size_t)j * F, 1, (size_t)F, sp))) != QKDREC_OK ||
                    (s = enq(cudaMemsetAsync(it_out + (size_t)j * F, 0, (size_t)F * 4, sp))) != QKDREC_OK)
                    break;
                continue;
            }
            const CodeDev &d = c->d;
            {
                // Bob's syndromes of slice j, 32 frames to a word (Sec. II Step 5)
                prof::Scope ps(prof::kSyndrome, sp);
                const int64_t tasks = W * (n / 16);
                pack_frames_kernel<<<(unsigned)std::min<int64_t>(ceil_div(tasks * 32, 256), (int64_t)sm_count() * 32),
                                     256, 0, sp>>>(bob + (size_t)j * count, n, F, W, bitsT);
                QKD_LAUNCHED("pack_frames_kernel");
                dim3 g((unsigned)ceil_div(d.M, 256), (unsigned)std::min<int64_t>(W, 65535));
                syndrome_packed_kernel<<<g, 256, 0, sp>>>(d.rp, d.ci, bitsT, n, d.M, W, W, sbits,
                                                          prof::counters(prof::kSyndrome));
                QKD_LAUNCHED("syndrome_packed_kernel");
            }
            // Alice: soft information of slice j from x and her reconciled lower slices
            if ((s = qkdrec_slice_llr(xd, count, m, j, lo, hi, sigma_n, label, j ? alice : nullptr, llr, spv)) !=
                QKDREC_OK)
                break;
            SyndIn si;
            si.packed = sbits;
            si.W = W;
            if ((s = decode_batch_impl(c, llr, si, F, opts, aj, it_out + (size_t)j * F, cv_out + (size_t)j * F,
                                       nullptr, slot + l.dec, l.dec_bytes, spv)) != QKDREC_OK)
                break;
        }
        if (s != QKDREC_OK) break;
        for (int32_t j = 0; j < m && s == QKDREC_OK; ++j)
            s = qkdrec_pack_bits(alice + (size_t)j * count, count, dev_a ? pt.alice_packed + j * plane8 : pk + j * plane8,
                                 spv);
        if (s == QKDREC_OK && !dev_a) s = put(pt.alice_packed, pk, (size_t)m * plane8, sp);
        if (s == QKDREC_OK && pt.converged && !dev_c) s = put(pt.converged, cv, (size_t)m * F, sp);
        if (s == QKDREC_OK && pt.iters && !dev_i) s = put(pt.iters, it, (size_t)m * F * 4, sp);
    }
    // join: the caller's stream waits for every side stream (also after an
    // error, so that no side stream is left forked)
    if (pool)
        for (int32_t k = 0; k < nslot; ++k) {
            QKD_CUDA(cudaEventRecord(pool->join[k], pool->st[k]));
            QKD_CUDA(cudaStreamWaitEvent(st, pool->join[k], 0));
        }
    return s;
}

}  // extern "C"

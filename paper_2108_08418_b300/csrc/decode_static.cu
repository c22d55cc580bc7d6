// qkdrec_decode_batch_static: the decoder run on a workspace that lives in a
// fixed device array compiled into the library, for callers that cannot
// allocate device memory themselves (see include/qkdrec.h).
#include <mutex>

#include "common.cuh"

namespace qkd {

// Workspace of the no-allocation decoder.  Every device that loads the
// library holds this array until the process exits; all calls share it.
constexpr size_t kStaticWorkspaceBytes = 32u << 20;
static __device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];

// The array's device address.  In host code the symbol is only a host-side
// stand-in, so the kernels get the address cudaGetSymbolAddress returns.  It
// is looked up again on every call made outside stream capture (a device
// reset reloads the module, and the array may move); a call made while its
// stream is capturing uses the address the last uncaptured call on that
// device found, so the first call on a device must come before any capture.
// Under lazy module loading the lookup is what loads the module, so the
// array's memory is committed at the first call on each device.
static std::mutex g_static_mu;
static void *g_static_ptr[64] = {nullptr};

static qkdrec_status static_workspace(cudaStream_t st, void **out) {
    int dev = 0;
    QKD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "device index %d above 63", dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    QKD_CUDA(cudaStreamIsCapturing(st, &cap));
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_workspace);
        if (e == cudaErrorMemoryAllocation)
            QKD_FAIL(QKDREC_ERR_NOMEM, "the built-in workspace (%zu bytes) could not be committed on device %d: %s",
                     kStaticWorkspaceBytes, dev, cudaGetErrorString(e));
        if (e != cudaSuccess || !p)
            QKD_FAIL(QKDREC_ERR_CUDA, "cudaGetSymbolAddress(static workspace): %s", cudaGetErrorString(e));
        g_static_ptr[dev] = p;
    } else if (!g_static_ptr[dev]) {
        QKD_FAIL(QKDREC_ERR_ARG, "first call on device %d made during stream capture; call once outside capture first",
                 dev);
    }
    *out = g_static_ptr[dev];
    return QKDREC_OK;
}

}  // namespace qkd

using namespace qkd;

extern "C" {

size_t qkdrec_decode_static_capacity(void) { return kStaticWorkspaceBytes; }

qkdrec_status qkdrec_decode_batch_static(qkdrec_code_t code, const float *llr, const uint8_t *synd, int32_t F,
                                         const qkdrec_decode_opts *opts, uint8_t *bits_out,
                                         int32_t *iters_out, uint8_t *conv_out, float *post_out,
                                         void *stream) {
    clear_error();
    if (!code) QKD_FAIL(QKDREC_ERR_ARG, "code is NULL");
    size_t need = 0;
    qkdrec_status s = qkdrec_decode_workspace_size(code, F, opts, &need);
    if (s != QKDREC_OK) return s;
    if (need > kStaticWorkspaceBytes)
        QKD_FAIL(QKDREC_ERR_ARG,
                 "decode needs %zu workspace bytes, above the %zu of the built-in workspace; "
                 "use fewer frames per call or qkdrec_decode_batch",
                 need, kStaticWorkspaceBytes);
    if (F == 0) return QKDREC_OK;
    void *ws = nullptr;
    if ((s = static_workspace(as_stream(stream), &ws)) != QKDREC_OK) return s;
    return qkdrec_decode_batch(code, llr, synd, F, opts, bits_out, iters_out, conv_out, post_out, ws,
                               kStaticWorkspaceBytes, stream);
}

}  // extern "C"

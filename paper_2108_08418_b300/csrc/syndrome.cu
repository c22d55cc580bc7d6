// Syndrome s = H b (mod 2) of F frames (Sec. II Step 5; Sec. III-B steps 2-3).
#include "common.cuh"
#include "profile.cuh"

namespace qkd {

// One thread per (check, frame): XOR of the frame's bits on the check's row.
// blockIdx.y walks frames, so the resident blocks gather from one frame's
// bit row (n bytes) and hit L1/L2.
__global__ void syndrome_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                const uint8_t *__restrict__ bits, int32_t n, int32_t M, int32_t F,
                                uint8_t *__restrict__ out, unsigned long long *prof) {
    unsigned long long units = 0, bytes = 0;
    for (int64_t f = blockIdx.y; f < F; f += gridDim.y) {
        const uint8_t *row = bits + f * n;
        for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < M; c += (int64_t)gridDim.x * blockDim.x) {
            uint32_t par = 0;
            const int32_t beg = __ldg(rp + c), end = __ldg(rp + c + 1);
            for (int32_t e = beg; e < end; ++e) par ^= __ldg(row + __ldg(ci + e));
            out[f * M + c] = (uint8_t)(par & 1u);
            ++units;
            bytes += (unsigned long long)(end - beg) + 1;   // bits gathered, syndrome bit written
        }
    }
    prof_add(prof, units, bytes);
}

}  // namespace qkd

using namespace qkd;

extern "C" qkdrec_status qkdrec_syndrome(qkdrec_code_t code, const uint8_t *bits, int32_t F, uint8_t *synd_out,
                                         void *stream) {
    clear_error();
    if (!code) QKD_FAIL(QKDREC_ERR_ARG, "code is NULL");
    if (F < 0) QKD_FAIL(QKDREC_ERR_ARG, "F < 0");
    if (F == 0) return QKDREC_OK;
    if (!bits || !synd_out) QKD_FAIL(QKDREC_ERR_ARG, "bits/synd_out NULL");
    const CodeDev &d = code->d;
    dim3 grid((unsigned)ceil_div(d.M, 256), (unsigned)(F < 65535 ? F : 65535));
    prof::Scope ps(prof::kSyndrome, as_stream(stream));
    syndrome_kernel<<<grid, 256, 0, as_stream(stream)>>>(d.rp, d.ci, bits, d.n, d.M, F, synd_out,
                                                         prof::counters(prof::kSyndrome));
    QKD_LAUNCHED("syndrome_kernel");
    return QKDREC_OK;
}

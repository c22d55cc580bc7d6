// Syndrome s = H b (mod 2) of F frames (Sec. II Step 5; Sec. III-B steps 2-3).
#include <algorithm>

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

// Bit planes of F frames in words of 32 frames: bits [F][n] (one byte per bit,
// n a multiple of 16, rows 16-byte aligned) -> bitsT [Wt][n] with bit f % 32 of
// bitsT[(f / 32) n + v] = bit v of frame f; frames F .. 32 Wt - 1 read as 0.
// One warp per (word, 16 variables): lane = frame, one 16-byte load per lane,
// 16 ballots, 16 consecutive words stored.
__global__ void pack_frames_kernel(const uint8_t *__restrict__ bits, int32_t n, int32_t F, int64_t Wt,
                                   uint32_t *__restrict__ bitsT) {
    const int lane = threadIdx.x & 31;
    const int64_t nchunk = n >> 4;
    const int64_t tasks = Wt * nchunk;
    const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tasks; t += wstride) {
        const int64_t w = t / nchunk, v0 = (t - w * nchunk) << 4;
        const int64_t f = (w << 5) + lane;
        uint4 b = make_uint4(0u, 0u, 0u, 0u);
        if (f < F) b = __ldg(reinterpret_cast<const uint4 *>(bits + f * n + v0));
        const uint32_t wd[4] = {b.x, b.y, b.z, b.w};
        uint32_t mine = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t word = __ballot_sync(0xffffffffu, (wd[k >> 2] >> ((k & 3) << 3)) & 1u);
            if (lane == k) mine = word;
        }
        if (lane < 16) bitsT[w * n + v0 + lane] = mine;
    }
}

// Syndromes of 32 frames at a time: sbits[c W + w] = XOR over the edges e of
// check c of bitsT[w n + ci[e]] (words w < Wt; the words up to W are 0).
// Thread per (check, word): a warp's checks gather from one row of bitsT.
__global__ void syndrome_packed_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                       const uint32_t *__restrict__ bitsT, int32_t n, int32_t M, int64_t Wt,
                                       int64_t W, uint32_t *__restrict__ sbits, unsigned long long *prof) {
    unsigned long long units = 0, bytes = 0;
    for (int64_t w = blockIdx.y; w < W; w += gridDim.y) {
        const uint32_t *row = bitsT + w * n;
        for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < M;
             c += (int64_t)gridDim.x * blockDim.x) {
            uint32_t par = 0;
            if (w < Wt) {
                const int32_t beg = __ldg(rp + c), end = __ldg(rp + c + 1);
                for (int32_t e = beg; e < end; ++e) par ^= __ldg(row + __ldg(ci + e));
                units += 32;
                bytes += 4ull * (end - beg) + 4;     // words gathered, syndrome word written
            }
            sbits[c * W + w] = par;
        }
    }
    prof_add(prof, units, bytes);
}

// Bits (one byte each, values 0/1) -> packed bytes, bit i % 8 of byte i / 8.
// Thread per 32 bits (two 16-byte loads, one word stored); count % 32 == 0.
__global__ void pack_bits_kernel(const uint8_t *__restrict__ bits, int64_t words, uint32_t *__restrict__ packed,
                                 unsigned long long *prof) {
    unsigned long long units = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 a = __ldg(reinterpret_cast<const uint4 *>(bits) + 2 * i);
        const uint4 b = __ldg(reinterpret_cast<const uint4 *>(bits) + 2 * i + 1);
        const uint32_t wd[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t out = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            // bytes of wd[k] hold bits 4k .. 4k + 3 in their lowest bit
            const uint32_t v = wd[k] & 0x01010101u;
            out |= ((v | (v >> 7) | (v >> 14) | (v >> 21)) & 0xFu) << (4 * k);
        }
        packed[i] = out;
        units += 32;
    }
    prof_add(prof, units, units + units / 8);
}

// Packed bytes -> one byte per bit (the inverse of pack_bits_kernel).
__global__ void unpack_bits_kernel(const uint32_t *__restrict__ packed, int64_t words, uint8_t *__restrict__ bits) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = __ldg(packed + i);
        uint32_t o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t q = (w >> (4 * k)) & 0xFu;
            o[k] = (q & 1u) | ((q & 2u) << 7) | ((q & 4u) << 14) | ((q & 8u) << 21);
        }
        reinterpret_cast<uint4 *>(bits)[2 * i] = make_uint4(o[0], o[1], o[2], o[3]);
        reinterpret_cast<uint4 *>(bits)[2 * i + 1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
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

extern "C" qkdrec_status qkdrec_pack_bits(const uint8_t *bits, int64_t count, uint8_t *packed, void *stream) {
    clear_error();
    if (count < 0 || count % 32) QKD_FAIL(QKDREC_ERR_ARG, "count=%lld must be a non-negative multiple of 32",
                                          (long long)count);
    if (count == 0) return QKDREC_OK;
    if (!bits || !packed) QKD_FAIL(QKDREC_ERR_ARG, "bits/packed NULL");
    if (reinterpret_cast<uintptr_t>(bits) % 16 || reinterpret_cast<uintptr_t>(packed) % 4)
        QKD_FAIL(QKDREC_ERR_ARG, "bits must be 16-byte and packed 4-byte aligned");
    const int64_t words = count / 32;
    prof::Scope ps(prof::kPack, as_stream(stream));
    pack_bits_kernel<<<(unsigned)std::min<int64_t>(ceil_div(words, 256), (int64_t)sm_count() * 16), 256, 0,
                       as_stream(stream)>>>(bits, words, reinterpret_cast<uint32_t *>(packed),
                                            prof::counters(prof::kPack));
    QKD_LAUNCHED("pack_bits_kernel");
    return QKDREC_OK;
}

extern "C" qkdrec_status qkdrec_unpack_bits(const uint8_t *packed, int64_t count, uint8_t *bits, void *stream) {
    clear_error();
    if (count < 0 || count % 32) QKD_FAIL(QKDREC_ERR_ARG, "count=%lld must be a non-negative multiple of 32",
                                          (long long)count);
    if (count == 0) return QKDREC_OK;
    if (!bits || !packed) QKD_FAIL(QKDREC_ERR_ARG, "bits/packed NULL");
    if (reinterpret_cast<uintptr_t>(bits) % 16 || reinterpret_cast<uintptr_t>(packed) % 4)
        QKD_FAIL(QKDREC_ERR_ARG, "bits must be 16-byte and packed 4-byte aligned");
    const int64_t words = count / 32;
    unpack_bits_kernel<<<(unsigned)std::min<int64_t>(ceil_div(words, 256), (int64_t)sm_count() * 16), 256, 0,
                         as_stream(stream)>>>(reinterpret_cast<const uint32_t *>(packed), words, bits);
    QKD_LAUNCHED("unpack_bits_kernel");
    return QKDREC_OK;
}

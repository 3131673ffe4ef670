// Host-side helpers shared by the tensor-core products of the plane and box paths:
// TF32 rounding of the precomputed operands, the persistent kernel's ring size and shared
// memory, and the K-major FP32 tensor maps its TMA loads read.
#pragma once
#include <cstring>
#include <vector>

#include "brs_internal.cuh"
#include "plane_tc.cuh"

namespace brs_tc {

// Round a value to TF32 (10 explicit mantissa bits), nearest with ties away from zero,
// the rounding of cvt.rna.tf32.f32.
inline float tf32_round(double x)
{
    float f = (float)x;
    uint32_t b;
    std::memcpy(&b, &f, 4);
    b = (b + 0x1000u) & 0xFFFFE000u;
    std::memcpy(&f, &b, 4);
    return f;
}

// Upload src split into TF32 hi = rn(x) and lo = rn(x - hi).
inline int upload_split(void** hi, void** lo, const std::vector<double>& src)
{
    std::vector<float> h(src.size()), l(src.size());
    for (size_t i = 0; i < src.size(); ++i) {
        h[i] = tf32_round(src[i]);
        l[i] = tf32_round(src[i] - (double)h[i]);
    }
    cudaError_t e = cudaMalloc(hi, h.size() * 4);
    if (e == cudaSuccess)
        e = cudaMemcpy(*hi, h.data(), h.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMalloc(lo, l.size() * 4);
    if (e == cudaSuccess)
        e = cudaMemcpy(*lo, l.data(), l.size() * 4, cudaMemcpyHostToDevice);
    return brs_cuda_status(e);
}

// Persistent products: ring stages per (split, tile N) so that the ring is 160-196 KB.
constexpr int pers_nst(int split, int bn)
{
    return bn == 256 ? (split == 3 ? 2 : 4)
                     : split == 3 ? (bn == 128 ? 3 : 4) : (bn == 128 ? 6 : 8);
}

// Ring stages of a persistent product with K blocks of bk FP32: as many as fit in 192 KB.
constexpr int ring_nst(int split, int bn, int bk)
{
    return (196608 / ((split == 3 ? 2 : 1) * (BM + bn) * bk * 4)) < 16
               ? 196608 / ((split == 3 ? 2 : 1) * (BM + bn) * bk * 4)
               : 16;
}

inline size_t pers_smem(int split, int bn, int nst = 0, int bk = BK)
{
    if (nst == 0)
        nst = pers_nst(split, bn);
    const size_t stage = (size_t)(split == 3 ? 2 : 1) * (BM + bn) * bk * 4;
    return 1024 + nst * stage + (2 * nst + 5) * 8 + 16;
}

// FP32 map with the K axis innermost, box (bk, box_rows[, 1]) with bk = 32 (128-byte swizzle)
// or 16 (64-byte swizzle); rank 3 when planes > 0.  K-major rows need kdim * 4 to be a
// multiple of 16 bytes.
inline int encode_map(CUtensorMap* m, const void* ptr, int kdim, int rows, int planes,
                      int box_rows, int bk = 32)
{
    PFN_encode_tiled fn = brs_encoder();
    if (!fn)
        return BRS_ERR_CUDA;
    if (bk != 16 && bk != 32)
        return BRS_ERR_ARG;
    cuuint64_t gdim[3] = {(cuuint64_t)kdim, (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t gstr[2] = {(cuuint64_t)kdim * 4, (cuuint64_t)kdim * rows * 4};
    cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)box_rows, 1u};
    cuuint32_t es[3] = {1u, 1u, 1u};
    const int rank = planes > 0 ? 3 : 2;
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<void*>(ptr), gdim, gstr,
                    box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    bk == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? BRS_OK : BRS_ERR_CUDA;
}

}  // namespace brs_tc

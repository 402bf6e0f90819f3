// Host packing of an operator for the tensor-core kernel (fr_gemm_tc.cu):
// split into bf16 hi = rn(a) and lo = rn(a - hi) (round to nearest even,
// from the float of the FP64 value), laid out in K-major core matrices.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "fr_kernels.h"

namespace fr {
namespace {

uint16_t bf16_rn(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    const uint32_t r = u + 0x7FFFu + ((u >> 16) & 1u);  // finite inputs only
    return (uint16_t)(r >> 16);
}

float bf16_to_float(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}

}  // namespace

void tc_pack(const double *A, int M, int K, std::vector<uint16_t> &img, int &Nmma, int &Kpad) {
    Nmma = (M + 15) / 16 * 16;
    Kpad = (K + 31) / 32 * 32;
    const size_t half = (size_t)Nmma * Kpad;  // elements of each of hi, lo
    img.assign(2 * half, 0);
    for (int i = 0; i < M; ++i)
        for (int k = 0; k < K; ++k) {
            const float a = (float)A[(size_t)i * K + k];
            const uint16_t hi = bf16_rn(a);
            const uint16_t lo = bf16_rn(a - bf16_to_float(hi));
            const int ks = k / 16, kk = k % 16;
            // byte offset / 2: K step block, core matrix (row group, K half), row, element
            const size_t off = (size_t)ks * Nmma * 16 + (size_t)((i / 8) * 2 + kk / 8) * 64 + (size_t)(i % 8) * 8 + kk % 8;
            img[off] = hi;
            img[half + off] = lo;
        }
}

}  // namespace fr

// Host packing of an operator for the tensor-core kernel (fr_gemm_tc.cu):
// split into bf16 hi = rn(a) and lo = rn(a - hi) (round to nearest even,
// from the float of the FP64 value), laid out in K-major core matrices; the
// columns of the two operand blocks (K1 from B1, K2 from B2) each start at a
// multiple of 16, so no 16-wide stage of K straddles B1 and B2.
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

void tc_pack(const double *A, int M, int K1, int K2, std::vector<uint16_t> &img, int &Nmma, int &K1pad, int &Kpad) {
    Nmma = (M + 15) / 16 * 16;
    K1pad = (K1 + 15) / 16 * 16;
    Kpad = K1pad + (K2 + 15) / 16 * 16;
    const int K = K1 + K2;
    const size_t half = (size_t)Nmma * Kpad;  // elements of each of hi, lo
    img.assign(2 * half, 0);
    for (int i = 0; i < M; ++i)
        for (int k = 0; k < K; ++k) {
            const float a = (float)A[(size_t)i * K + k];
            const uint16_t hi = bf16_rn(a);
            const uint16_t lo = bf16_rn(a - bf16_to_float(hi));
            // the columns of the second block start at a 16-column boundary
            const int kc = k < K1 ? k : K1pad + (k - K1);
            const int ks = kc / 16, kk = kc % 16;
            // byte offset / 2: K step block, core matrix (row group, K half), row, element
            const size_t off = (size_t)ks * Nmma * 16 + (size_t)((i / 8) * 2 + kk / 8) * 64 + (size_t)(i % 8) * 8 + kk % 8;
            img[off] = hi;
            img[half + off] = lo;
        }
}

}  // namespace fr

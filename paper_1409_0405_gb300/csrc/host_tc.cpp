// Host packing of an operator for the tensor-core kernel (fr_gemm_tc.cu):
// split into bf16 hi = rn(a) and lo = rn(a - hi) (round to nearest even,
// from the float of the FP64 value), laid out in K-major core matrices; the
// columns of the two operand blocks (K1 from B1, K2 from B2) each start at a
// multiple of 16, so no 16-wide stage of K straddles B1 and B2.  The split
// TF32 image (hi = tf32(a), lo = tf32(a - hi)) is laid out stage by stage,
// so that one contiguous slab per stage can be copied next to the state.
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

// FP32 -> TF32 (10 stored mantissa bits), round half away from zero, the
// low 13 bits cleared (the device converter rounds the same way)
uint32_t tf32_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return (u + 0x1000u) & 0xFFFFE000u;
}

float bits_to_float(uint32_t u) {
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}

}  // namespace

void tc_pack_tf32(const double *A, int M, int K1, int K2, std::vector<uint32_t> &img, int &Nmma, int &K1pad,
                  int &Kpad) {
    Nmma = (M + 15) / 16 * 16;
    K1pad = (K1 + 15) / 16 * 16;
    Kpad = K1pad + (K2 + 15) / 16 * 16;
    const int K = K1 + K2;
    const size_t slab = (size_t)Nmma * 16 * 2;  // values per stage (hi and lo)
    img.assign(slab * (Kpad / 16), 0u);
    for (int i = 0; i < M; ++i)
        for (int k = 0; k < K; ++k) {
            const float a = (float)A[(size_t)i * K + k];
            const uint32_t hi = tf32_bits(a);
            const uint32_t lo = tf32_bits(a - bits_to_float(hi));
            const int kc = k < K1 ? k : K1pad + (k - K1);
            const int ks = kc / 16, kk = kc % 16;
            // stage ks; row group i/8, K core matrix kk/4, row i%8, value kk%4
            const size_t off = (size_t)ks * slab + (size_t)(i / 8) * 128 + (size_t)(kk / 4) * 32 + (size_t)(i % 8) * 4 + kk % 4;
            img[off] = hi;
            img[off + (size_t)Nmma * 16] = lo;
        }
}

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

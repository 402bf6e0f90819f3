// Host packing of an FP64 operator for the exact-split tensor-core kernel
// (fr_gemm_x64.cu, FR_FP64S): per operator row the largest biased exponent
// E, and the eight signed base-128 digits of X = round(a 2^(56 - (E - 1022)))
// of every entry a, each digit as a bf16 (exact: |d| <= 128), laid out per
// row block and 16-wide K stage in the K-major core-matrix layout of the
// MMA's B operand.  The device converter splits the state the same way
// (with per-column exponents).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "fr_kernels.h"

namespace fr {
namespace {

// the biased exponent field, 1 for a subnormal, 0 for zero
int exp_field(double x) {
    uint64_t b;
    std::memcpy(&b, &x, 8);
    const int be = (int)((b >> 52) & 0x7FF);
    if (be) return be;
    return (b << 1) ? 1 : 0;
}

// X = round(x 2^(56 - (E - 1022))) for |x| < 2^(E - 1022) (half away from
// zero), as the device converter computes it
int64_t fixed56(double x, int E) {
    uint64_t b;
    std::memcpy(&b, &x, 8);
    int be = (int)((b >> 52) & 0x7FF);
    uint64_t m = b & 0xFFFFFFFFFFFFFull;
    if (be) m |= 1ull << 52;
    else be = 1;
    const int s = be - E + 3;
    uint64_t X;
    if (s >= 0) X = m << s;
    else if (s > -54) X = (m + (1ull << (-s - 1))) >> (-s);
    else X = 0;
    return (b >> 63) ? -(int64_t)X : (int64_t)X;
}

uint16_t bf16_of_int(int d) {
    const float f = (float)d;  // |d| <= 128: exact, and exact in bf16
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

}  // namespace

// the digits d_0..d_7 of X: Y = X + 64 (128^6 + ... + 1); d_0 = floor(Y /
// 128^7), d_p = ((Y >> 7 (7 - p)) & 127) - 64
void x64_digits(int64_t X, int d[kX64Digits]) {
    constexpr int64_t kOff = 64ll * ((1ll << 42) + (1ll << 35) + (1ll << 28) + (1ll << 21) + (1ll << 14) + (1ll << 7) + 1ll);
    const int64_t Y = X + kOff;
    d[0] = (int)(Y >> 49);  // arithmetic shift: floor
    for (int p = 1; p < kX64Digits; ++p) d[p] = (int)((Y >> (7 * (7 - p))) & 127) - 64;
}

bool x64_pack(const double *A, int M, int K1, int K2, bool mult3, std::vector<uint16_t> &img,
              std::vector<int> &rexp, X64Operator &op) {
    const int K = K1 + K2;
    if (M <= 0 || K <= 0 || K > kX64MaxK) return false;
    op.M = M;
    op.K1 = K1;
    op.K2 = K2;
    op.K1pad = (K1 + 15) / 16 * 16;
    op.Kpad = op.K1pad + (K2 + 15) / 16 * 16;
    // row blocks of at most 64 rows, as even as possible (whole points)
    const int unit = mult3 ? 3 : 1;
    op.nrb = (M + kX64MaxRows - 1) / kX64MaxRows;
    int rows = (M + op.nrb - 1) / op.nrb;
    rows = (rows + unit - 1) / unit * unit;
    while (rows > kX64MaxRows) rows -= unit;
    op.nrb = (M + rows - 1) / rows;
    op.rows = rows;
    op.Nmma = (rows + 15) / 16 * 16;
    op.wide = 0;
    for (int L = 0; L < kX64Digits; ++L) {
        const int64_t bound = L == 0 ? (int64_t)K << 14 : ((int64_t)K << 12) * (L + 3);
        if (bound >= (1ll << 22)) op.wide |= 1u << L;
    }
    rexp.assign((size_t)M, 0);
    for (int i = 0; i < M; ++i)
        for (int k = 0; k < K; ++k) {
            const int e = exp_field(A[(size_t)i * K + k]);
            if (e > rexp[(size_t)i]) rexp[(size_t)i] = e;
        }
    const int nks = op.Kpad / 16;
    const size_t slab = (size_t)op.Nmma * 16;  // bf16 values of one digit's stage slab
    img.assign((size_t)op.nrb * nks * kX64Digits * slab, 0);
    for (int i = 0; i < M; ++i) {
        if (!rexp[(size_t)i]) continue;
        const int rb = i / rows, il = i - rb * rows;
        for (int k = 0; k < K; ++k) {
            int d[kX64Digits];
            x64_digits(fixed56(A[(size_t)i * K + k], rexp[(size_t)i]), d);
            const int kc = k < K1 ? k : op.K1pad + (k - K1);
            const int ks = kc / 16, kk = kc % 16;
            // core matrix (row group, K half), row within it, value
            const size_t in_slab = (size_t)((il / 8) * 2 + kk / 8) * 64 + (size_t)(il % 8) * 8 + kk % 8;
            for (int q = 0; q < kX64Digits; ++q)
                img[(((size_t)rb * nks + ks) * kX64Digits + q) * slab + in_slab] = bf16_of_int(d[q]);
        }
    }
    return true;
}

}  // namespace fr

// Bit-pattern helpers of the split (Ozaki) path, shared by the density's evaluation kernel
// (which reduces the point exponents while it produces the values) and the slicing kernels
// (which turn the values into digits).
//
// On this GPU the FP64 pipe is ~1/60 of the FP32 rate, so exponents are taken from FP64 bit
// patterns with integer and FP32 instructions rather than from FP64 products.
#pragma once

#ifdef __CUDACC__
#include "nao_internal.h"

namespace split_bits {

// |x| as an ordered integer: for non-negative doubles the bit patterns order like the values.
__device__ __forceinline__ long long abs_bits(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL; }

// The biased exponent field of the FP64 with bit pattern xb.
__device__ __forceinline__ int biased_exponent(long long xb) { return (int)((xb >> 52) & 0x7FF); }

// The significand of the FP64 with bit pattern xb, in [1, 2), truncated to FP32.
__device__ __forceinline__ float significand_f(long long xb) {
    return __int_as_float(0x3F800000 | (int)((xb >> 29) & 0x7FFFFF));
}

// Exponent e with max * 2^-e in [0.25, 0.5), from the biased exponent eb of max; rows whose
// magnitude is below 2^-900 (or zero, eb = 0) are taken as zero (flag -10000).
__device__ __forceinline__ int exponent_of_binade(int eb) {
    if (eb <= 0) return -10000;
    const int ex = eb - 1022;  // max = f 2^ex, f in [0.5, 1)
    return ex < -900 ? -10000 : ex + 1;
}

// d_k of the Hamiltonian's column k = (component c, batch-ordered point p): w v on the potential
// part (c = 0), w (kappa + v_tau) / 2 on the three gradient parts (Eq. H_decomp; kappa = 1 with
// the kinetic term, v_tau with the meta-GGA term), 0 for a term that is off; the column's scale
// is sqrt|d_k| (formed in the H slicer).
__device__ __forceinline__ double h_column_weight(const DevSystem &s, int m, int p, int c, uint32_t terms) {
    const double w = s.pw[p];
    if (c == 0) return (terms & NAO_TERM_POTENTIAL) ? w * v_at(s, m, p) : 0.0;
    const double kin = (terms & NAO_TERM_KINETIC) ? 1.0 : 0.0;
    return 0.5 * w * ((terms & NAO_TERM_TAU) ? kin + vt_at(s, m, p) : kin);
}

// Ordering key of |x sd| for the row maximum without an FP64 product: the product's biased
// exponent is eb(x) + eb(sd) - 1023, plus 1 when the significands' product reaches 2 (taken as
// reached from 2 - 2^-20 on, since both significands are truncated to FP32: the exponent may
// then be one too large, costing one bit, but never too small). 0 for a zero or subnormal
// factor. ebs, ms: biased exponent and significand_f of sd.
__device__ __forceinline__ int h_row_key(double x, int ebs, float ms) {
    const long long xb = __double_as_longlong(x);
    const int ebx = biased_exponent(xb);
    if (ebx == 0 || ebs == 0) return 0;
    return ebx + ebs + (significand_f(xb) * ms >= 1.999998f ? 1 : 0);
}

// The same key for a float-float factor x = h + l given by its high part h (FP32): the exponent
// of h on the FP64 scale, and the threshold lowered to 2 - 2^-13 so that the low parts of x and
// of sd (a few 2^-24 relative) cannot carry the product into the next binade unnoticed.
__device__ __forceinline__ int h_row_key_ff(float xh, int ebs, float ms) {
    const int xb = __float_as_int(xh);
    const int ebx = (xb >> 23) & 0xFF;
    if (ebx == 0 || ebs == 0) return 0;
    const float sx = __int_as_float(0x3F800000 | (xb & 0x7FFFFF));
    return ebx + 896 + ebs + (sx * ms >= 1.99988f ? 1 : 0);
}

// Row exponent from the maximum key of the row.
__device__ __forceinline__ int h_row_exponent(int mk) { return exponent_of_binade(mk - 1023); }

}  // namespace split_bits
#endif

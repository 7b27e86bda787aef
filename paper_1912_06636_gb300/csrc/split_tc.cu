// Split-precision (Ozaki) contractions on the tcgen05 tensor cores.
//
// The batch products of Eq. batch_matrix_mult (Hamiltonian) and of the density (Eq. Density
// restricted to nnz(B)) are dense matrix products whose inputs are FP64. Each input row x
// (one basis function over the batch's points for H; one point over the basis for n; one
// density-matrix row for n) is scaled by a power of two 2^-e so that |x 2^-e| < 1/2, rounded
// to an integer X = round(x 2^(6S-e)) and cut into S balanced base-64 digits
//     X = sum_s d_s 64^(S-1-s),  d_s in [-32, 32],
// (Ozaki, Ogita, Oishi, Rump, "Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication", Numer. Algorithms 59 (2012): a splitting whose
// slice products are exact in the working precision of the fast product). Every digit is an
// exact bf16 integer, every digit product is at most 2^10, and a K-long sum of the products of
// one slice-order group g = s + t (g + 1 pairs) stays below K (g+1) 2^10 < 2^24, so it is exact
// in the FP32 accumulator. Each group therefore has its own accumulator in tensor memory;
// pairs with s + t >= S are dropped (their weight is below 64^-S). The epilogue recombines the
// groups as integers (three 64-bit parts) and scales once in FP64:
//     x_i . y_j = 2^(e_i + e_j) sum_g M_g 64^-(g+2).
// Tensor memory holds S groups x TN columns: TN = 48 for S <= 10, TN = 32 for S = 11, 12.
//
// Hamiltonian: A = F (rows i, K = 4 Ppad: phi | d/dx | d/dy | d/dz weighted by sqrt|d_k|) and
// B = sign(d_k) F (rows j), tiles of 128 x TN (S groups x TN FP32 columns, at most 480 of the
// 512 tensor-memory columns), tile pairs crossing the upper triangle, FP64 atomic scatter.
// Density: A = Phi^T (rows = points, K = basis), B = P' (rows j, P'_ij = c_IJ P_ij for TN-function
// tiles I <= J with c_II = 1, c_IJ = 2, else 0) so that T_qj = sum_i phi_qi P'_ij and
// n_q = sum_j T_qj phi_qj; one per-batch exponent is used for P'.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "ff.h"
#include "nao_internal.h"
#include "split_bits.h"
#include "tc_ptx.h"

namespace {

constexpr long long kWaitCycles = 400000000LL;  // ~0.2 s at 2 GHz: bounded mbarrier waits


// Digit extraction works on FP64 bit patterns with integer instructions: on this GPU the FP64
// pipe is ~1/60 of the FP32 rate, and a double-to-int64 conversion per element would make the
// slicing kernels FP64-bound.
using split_bits::abs_bits;

// S balanced base-2^B digits (B = 6: base 64, |d| <= 32, bf16; B = 5: base 32, |d| <= 16, e4m3;
// most significant first in dig[0]) of X = round(x 2^(BS-e)), |x 2^-e| < 1/2, as exact
// small-integer floats. From x's bits x = +-m 2^(E-1075) (53-bit m): |X| = m 2^-sh with
// sh = 1075 + e - BS - E, rounded half up when sh > 0, held as a 128-bit integer (hi:lo; more
// than 64 bits only for BS > 64). |X| is cut into chunks of D digits (3 x 6 = 18 or 4 x 5 = 20
// bits; the fourth chunk takes the remaining 23 bits), exact in FP32, and the digits are peeled
// off from the bottom in FP32: q = rint(v / 2^B), d = v - 2^B q in [-2^(B-1), 2^(B-1)], v <- q,
// the carry q (0 or 1 after a chunk's digits) joining the next chunk. The top digit keeps
// whatever remains, which the bound on |X| keeps in range. Subnormal x and e = -10000 give zeros.
// |X| = round(|x| 2^(BS-e)) as a 128-bit integer (hi:lo) from the bits of x, and the sign of x.
template <int S, int B>
__device__ __forceinline__ void digit_integer(double x, int e, unsigned long long &lo, unsigned long long &hi,
                                              float &sgn) {
    const long long bits = __double_as_longlong(x);
    const int eb = (int)((bits >> 52) & 0x7FF);
    lo = 0;
    hi = 0;
    if (eb != 0 && e > -10000) {
        const unsigned long long m = ((unsigned long long)bits & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
        const int sh = 1075 + e - B * S - eb;
        if (sh > 0) {
            lo = sh >= 63 ? 0ULL : (m + (1ULL << (sh - 1))) >> sh;
        } else {
            const int k = -sh;  // <= B S - 54: 18 for 12 bf16 slices, 26 for 16 e4m3 slices
            lo = m << k;
            hi = k > 0 ? m >> (64 - k) : 0ULL;
        }
    }
    sgn = bits < 0 ? -1.0f : 1.0f;
}

// Chunk c of |X| = (hi:lo): c = 0, 1, 2 the CB-bit fields (CB = 3 x 6 or 4 x 5 bits), c = 3 the
// 23 bits from bit 3 CB.
template <int B>
__device__ __forceinline__ uint32_t digit_chunk(unsigned long long lo, unsigned long long hi, int c) {
    constexpr int CB = B == 6 ? 18 : 20;
    constexpr unsigned long long M = (1ULL << CB) - 1;
    return c == 0 ? (uint32_t)(lo & M)
         : c == 1 ? (uint32_t)((lo >> CB) & M)
         : c == 2 ? (uint32_t)((lo >> (2 * CB)) & M)
                  : (uint32_t)(((lo >> (3 * CB)) | (hi << (64 - 3 * CB))) & 0x7FFFFFULL);
}

// The S digits of two values x0, x1 at once (.x and .y of dig[s]) with packed FP32x2 arithmetic.
// The sign is carried in the running value: v starts as sgn (|X| mod 2^CB) (sgn (2^23 + u) - sgn 2^23,
// one packed FMA, exact), every later chunk enters as + sgn u at its digit position, and the
// peeling q = rint(v / 2^B), d = v - 2^B q works on signed v as well: rint is odd-symmetric, so
// the digits are those of |X| times the sign.
template <int S, int B>
__device__ __forceinline__ void digits2(double x0, double x1, int e, float2 (&dig)[S]) {
    constexpr int D = B == 6 ? 3 : 4;  // digits per chunk
    unsigned long long lo0, hi0, lo1, hi1;
    float s0, s1;
    digit_integer<S, B>(x0, e, lo0, hi0, s0);
    digit_integer<S, B>(x1, e, lo1, hi1, s1);
    const float2 sgn = make_float2(s0, s1), nb = make_float2(-8388608.0f * s0, -8388608.0f * s1);
    const float2 inv = make_float2(1.0f / (1 << B), 1.0f / (1 << B)), big = make_float2(12582912.0f, 12582912.0f);
    const float2 nbig = make_float2(-12582912.0f, -12582912.0f), mb = make_float2(-(float)(1 << B), -(float)(1 << B));
    auto chunk = [&](int c) {  // sgn u, u < 2^23, exactly
        const float2 u = make_float2(__int_as_float(0x4B000000 | (int)digit_chunk<B>(lo0, hi0, c)),
                                     __int_as_float(0x4B000000 | (int)digit_chunk<B>(lo1, hi1, c)));
        return __ffma2_rn(sgn, u, nb);
    };
    float2 v = chunk(0);
#pragma unroll
    for (int s = S - 1; s >= 0; s--) {
        const int t = S - 1 - s;  // digits already taken
        if (t > 0 && t % D == 0) v = __fadd2_rn(v, chunk(t / D));
        if (s == 0) {
            dig[0] = v;
        } else {
            const float2 q = __fadd2_rn(__ffma2_rn(v, inv, big), nbig);  // rint(v / 2^B)
            dig[s] = __ffma2_rn(q, mb, v);
            v = q;
        }
    }
}

// The digits of a float-float value without 128-bit integers: x = h + l is scaled by 2^(BS-e)
// through its exponent fields (H = h 2^(BS-e), L = l 2^(BS-e), exact), and each part is cut into
// balanced chunks of CB bits from the top in FP32: q = rint(R 2^-(c CB)), R <- R - q 2^(c CB),
// for c = 3, 2, 1, then u_0 = rint(R). Every step is exact (R keeps a subset of the part's 24
// significand bits; |R 2^-(c CB)| < 2^22 keeps the rounding by 1.5 2^23 valid), so
// sum_c u_c 2^(c CB) = round(H) and the chunks of round(H) + round(L), summed per chunk (each at
// most 2^(CB-1) in magnitude), feed the digit peeling below; the result is within one unit of
// round(|h + l| 2^(BS-e)). A part below the FP32 normal range after scaling counts as zero.
__device__ __forceinline__ float ff_scale_pow2(float v, int k) {
    const int b = __float_as_int(v);
    const int ex = (b >> 23) & 0xFF;
    if (ex == 0 || ex + k <= 0) return 0.0f;
    return __int_as_float(b + (k << 23));
}

__device__ __forceinline__ float rint_small(float y) {  // |y| < 2^22
    return __fsub_rn(__fadd_rn(y, 12582912.0f), 12582912.0f);
}

template <int CB>
__device__ __forceinline__ void ff_part_chunks(float P, float (&u)[4]) {
    constexpr float W1 = (float)(1ULL << CB), W2 = W1 * W1, W3 = W2 * W1;
    constexpr float I1 = 1.0f / W1, I2 = I1 * I1, I3 = I2 * I1;
    float R = P;
    const float q3 = rint_small(__fmul_rn(R, I3));
    R = __fmaf_rn(-q3, W3, R);
    const float q2 = rint_small(__fmul_rn(R, I2));
    R = __fmaf_rn(-q2, W2, R);
    const float q1 = rint_small(__fmul_rn(R, I1));
    R = __fmaf_rn(-q1, W1, R);
    u[0] += rint_small(R);
    u[1] += q1;
    u[2] += q2;
    u[3] += q3;
}

template <int S, int B>
__device__ __forceinline__ void ff_chunks(ffa::F x, int e, float (&u)[4]) {
    constexpr int D = B == 6 ? 3 : 4, CB = D * B;
    u[0] = u[1] = u[2] = u[3] = 0.0f;
    if (e <= -10000) return;
    const int k = B * S - e;
    ff_part_chunks<CB>(ff_scale_pow2(x.h, k), u);
    ff_part_chunks<CB>(ff_scale_pow2(x.l, k), u);
}

// The S digits of two float-float values at once (packed FP32x2 peeling, as for FP64 values).
template <int S, int B>
__device__ __forceinline__ void digits2(ffa::F x0, ffa::F x1, int e, float2 (&dig)[S]) {
    constexpr int D = B == 6 ? 3 : 4;
    float u0[4], u1[4];
    ff_chunks<S, B>(x0, e, u0);
    ff_chunks<S, B>(x1, e, u1);
    const float2 inv = make_float2(1.0f / (1 << B), 1.0f / (1 << B)), big = make_float2(12582912.0f, 12582912.0f);
    const float2 nbig = make_float2(-12582912.0f, -12582912.0f), mb = make_float2(-(float)(1 << B), -(float)(1 << B));
    float2 v = make_float2(u0[0], u1[0]);
#pragma unroll
    for (int s = S - 1; s >= 0; s--) {
        const int t = S - 1 - s;
        if (t > 0 && t % D == 0) v = __fadd2_rn(v, make_float2(u0[t / D], u1[t / D]));
        if (s == 0) {
            dig[0] = v;
        } else {
            const float2 q = __fadd2_rn(__ffma2_rn(v, inv, big), nbig);
            dig[s] = __ffma2_rn(q, mb, v);
            v = q;
        }
    }
}

// bf16 bit patterns of two small integers held exactly in floats (their low halves are zero).
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

// e4m3 bytes of four integers |d| <= 16 held in floats (each exact in e4m3), a at the lowest
// address. cvt...e4m3x2 puts its first source in the upper byte of the pair.
__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d) {
    unsigned short lo, hi;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(b), "f"(a));
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(d), "f"(c));
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

// Digits of the 128-byte row segment a lane owns in one K chunk: values x[0..LC-1] of its LC
// columns (2 for bf16, 4 for e4m3; FP64 or float-float), packed per slice into one 32-bit word.
template <int S, int F, typename V>
__device__ __forceinline__ void lane_digit_words(const V *x, int e, uint32_t (&w)[S]) {
    constexpr int B = nao_digit_bits(F);
    float2 d0[S];
    digits2<S, B>(x[0], x[1], e, d0);
    if constexpr (F == NAO_DIGITS_BF16) {
#pragma unroll
        for (int sl = 0; sl < S; sl++) w[sl] = pack_bf16x2(d0[sl].x, d0[sl].y);
    } else {
        float2 d1[S];
        digits2<S, B>(x[2], x[3], e, d1);
#pragma unroll
        for (int sl = 0; sl < S; sl++) w[sl] = pack_e4m3x4(d0[sl].x, d0[sl].y, d1[sl].x, d1[sl].y);
    }
}

// 2^E as an FP64 (0 below the normal range).
__device__ __forceinline__ double pow2(int E) {
    if (E < -1022) return 0.0;
    if (E > 1023) E = 1023;
    return __longlong_as_double((long long)(1023 + E) << 52);
}


// ----------------------------------------------------------------------------------------
// Hamiltonian slicing: one CTA per (batch, 64-row tile of basis functions). Columns are
// reordered: the negative-weight ones (v < 0 on the potential part) first, padded to a whole
// MMA K step (16 bf16 or 32 e4m3 columns), then the rest, so that B = A and the sign is applied
// per K step.
// One warp per row: the row's exponent (a pass over the row's K float-float values), then its
// digits (a second pass, served from L2: the slices are written with evict-first stores so that
// they do not push the rows out). Within each K step, lane l of the 8 lanes that write the
// step's 32 bytes takes logical columns l, l + 8 (, l + 16, l + 24) of the step: a permutation
// inside the K step, the same for every row (A and B of H are the same digit rows, so every
// product is unchanged, and each K step keeps its sign), which keeps each load instruction of the
// second pass on a few 64-byte runs of the row.
// ----------------------------------------------------------------------------------------
template <int S, int F>
__global__ void __launch_bounds__(256, S <= 10 ? 5 : 4) slice_h_kernel(DevSystem s, int32_t b0, const FF2 *__restrict__ scratch,
                                                        uint32_t terms, uint8_t *__restrict__ slices,
                                                        const int64_t *__restrict__ sl_off, int32_t *__restrict__ expo,
                                                        int32_t *__restrict__ neg16) {
    __shared__ ffa::F sd[4 * NAO_SPLIT_MAX_PPAD];    // column scale as a float-float
    __shared__ int sd_eb[4 * NAO_SPLIT_MAX_PPAD];    // biased exponent of sd (0: zero weight)
    __shared__ float sd_m[4 * NAO_SPLIT_MAX_PPAD];   // significand of sd in [1, 2)
    __shared__ short src[4 * NAO_SPLIT_MAX_PPAD + 128];
    __shared__ unsigned char negf[4 * NAO_SPLIT_MAX_PPAD];
    __shared__ int wsum[8];
    const int b = b0 + blockIdx.x, rt = blockIdx.y, m = s.sys.bmol[b];
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    constexpr int C = nao_chunk_cols(F), KS = nao_kstep_cols(F), LC = C / 32;  // columns per lane
    const SplitGeom G(P, N, S, 0, F);
    if (N == 0 || rt >= G.h_slice_tiles()) return;
    const int K = 4 * Ppad, Kp = C * G.n_kc;
    const FF2 *E = scratch + s.scr_off[b];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const int c = k / Ppad, q = k - c * Ppad;
        const double d = q < P ? split_bits::h_column_weight(s, m, p0 + q, c, terms) : 0.0;
        // sqrt|d| as a float-float: the FP32 square root s0 and one Newton correction
        // (|d| - s0^2) / (2 s0), the residual formed exactly by one FP64 FMA (|d| below the FP32
        // range counts as a zero weight)
        const float a = __double2float_rn(fabs(d));
        ffa::F sdf{0.0f, 0.0f};
        if (a >= 1.17549435e-38f) {
            const float s0 = __fsqrt_rn(a);
            const double r = fma(-(double)s0, (double)s0, fabs(d));
            sdf = ffa::quick(s0, __fmul_rn(__double2float_rn(r), __fdiv_rn(0.5f, s0)));
        }
        sd[k] = sdf;
        const int sb = __float_as_int(sdf.h);
        sd_eb[k] = sdf.h != 0.0f ? ((sb >> 23) & 0xFF) + 896 : 0;  // biased exponent on the FP64 scale
        sd_m[k] = __int_as_float(0x3F800000 | (sb & 0x7FFFFF));
        negf[k] = d < 0.0 ? 1 : 0;
    }
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) src[k] = -1;
    __syncthreads();
    // exclusive scan of the negative flags: thread t owns columns [t*per, t*per + per)
    const int per = (K + 255) / 256;
    const int kb = threadIdx.x * per, ke = min(K, kb + per);
    int cnt = 0;
    for (int k = kb; k < ke; k++) cnt += negf[k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < 8; w++) {
        if (w < warp) before += wsum[w];
        total += wsum[w];
    }
    before += incl - cnt;
    const int negpad = (total + KS - 1) / KS * KS;  // a whole MMA K step
    for (int k = kb; k < ke; k++) {
        const int pos = negf[k] ? before : negpad + k - before;
        before += negf[k];
        src[pos] = (short)k;
    }
    if (rt == 0 && threadIdx.x == 0) neg16[b] = negpad / KS;  // negated K steps
    __syncthreads();
    uint8_t *base = slices + sl_off[b];
    // the logical column of this lane's value c inside a chunk (see above)
    const int lcol = KS * (lane >> 3) + (lane & 7);
    for (int lr = warp; lr < 64; lr += 8) {
        const int r = rt * 64 + lr;
        if (r >= G.R16) break;
        const float2 *row = reinterpret_cast<const float2 *>(E + (int64_t)(r < N ? r : 0) * K);
        int mk = 0;
        if (r < N)
            for (int k = lane; k < K; k += 32) mk = max(mk, split_bits::h_row_key_ff(row[k].x, sd_eb[k], sd_m[k]));
        mk = __reduce_max_sync(0xffffffffu, mk);
        const int e = r < N ? split_bits::h_row_exponent(mk) : -10000;
        if (lane == 0 && r < N) expo[s.rel_off[b] + r] = e;
        for (int kc = 0; kc < G.n_kc; kc++) {
            ffa::F x[LC];
#pragma unroll
            for (int c = 0; c < LC; c++) {
                const int kk = src[C * kc + lcol + 8 * c];
                if (kk >= 0 && e > -10000) {
                    const float2 v = __ldcs(row + kk);
                    x[c] = ffa::mul(ffa::F{v.x, v.y}, sd[kk]);
                } else {
                    x[c] = ffa::F{0.0f, 0.0f};
                }
            }
            uint32_t wd[S];
            lane_digit_words<S, F>(x, e, wd);
            const uint32_t off = tc::sw128_byte((uint32_t)r, (uint32_t)(4 * lane));
#pragma unroll
            for (int sl = 0; sl < S; sl++) __stcs(reinterpret_cast<unsigned int *>(base + G.h_block(sl, kc) + off), wd[sl]);
        }
    }
}

// ----------------------------------------------------------------------------------------
// Density slicing.
// Phi^T: one CTA (8 warps) per (batch, 32-point tile), the point exponents from the
// evaluation. Per K chunk (64 or 128 functions) the CTA stages phi[i][q] (chunk x 32, read along
// the points) in shared memory and each warp writes its points' rows along K (2 or 4 functions
// per lane, one 128-byte row segment per slice). CTAs with blockIdx.y = 0 instead reduce the batch's
// exponent of P' (the upper-triangle tile pairs, read along rows of P).
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ int tile_of(int i, int TN) { return i / TN; }

template <typename V>
struct StageOf {  // shared-memory staging type of the density slicer's input
    using type = ffa::F;
    __device__ static ffa::F get(const FF2 &v) { return v.f(); }
    __device__ static ffa::F zero() { return ffa::F{0.0f, 0.0f}; }
};
template <>
struct StageOf<double> {
    using type = double;
    __device__ static double get(double v) { return v; }
    __device__ static double zero() { return 0.0; }
};

// V = FF2: the split path's float-float phi (rows of ld_mult Ppad at scr_off[b]); V = double: the
// density Hessian's FP64 evaluation (rows of 10 Ppad at eoff[b]), component row coff (phi or one
// gradient component). pexp = 0 leaves the P' exponent (blockIdx.y = 0) to another launch.
template <int S, int F, typename V>
__global__ void __launch_bounds__(256) slice_nphi_kernel(DevSystem s, int32_t b0, const V *__restrict__ scratch,
                                                        const int64_t *__restrict__ eoff, int coff,
                                                        uint8_t *__restrict__ slices, const int64_t *__restrict__ sl_off,
                                                        const int32_t *__restrict__ expo_q, int32_t *__restrict__ expo_b,
                                                        const int32_t *__restrict__ tn_b, int ld_mult, int full, int pexp) {
    constexpr int C = nao_chunk_cols(F), LC = C / 32;
    using TT = typename StageOf<V>::type;
    __shared__ TT t[32][C + 1];
    __shared__ int red[8];
    const int b = b0 + blockIdx.x;
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    if (N == 0) return;
    const SplitGeom G(P, N, S, 0, F);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.y == 0) {
        if (!pexp) return;
        // max |P'_ij| over i <= j (P' is P on the diagonal tiles, 2 P off them, 0 below unless
        // full): the exponent field of |P| plus one off the diagonal tiles
        const int m = s.sys.bmol[b], TN = tn_b[b];
        const int32_t *rel = s.rel_idx + s.rel_off[b];
        int mk = 0;
        for (int i = warp; i < N; i += 8) {
            const int64_t gi = rel[i];
            for (int j = (full ? 0 : i) + lane; j < N; j += 32) {
                const int64_t gj = rel[j];
                const int eb = split_bits::biased_exponent(abs_bits(gi <= gj ? p_elem(s, m, gi, gj) : p_elem(s, m, gj, gi)));
                if (eb != 0) mk = max(mk, eb + ((!full && tile_of(i, TN) < tile_of(j, TN)) ? 1 : 0));
            }
        }
        mk = __reduce_max_sync(0xffffffffu, mk);
        if (lane == 0) red[warp] = mk;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < 8; w++) mk = max(mk, red[w]);
            expo_b[b] = split_bits::exponent_of_binade(mk);
        }
        return;
    }
    const int q0 = (blockIdx.y - 1) * 32;
    if (q0 >= G.P16) return;
    const V *E = scratch + eoff[b] + (int64_t)coff * Ppad;  // row i at E + i ld_mult Ppad
    const int64_t ld = (int64_t)ld_mult * Ppad;
    const bool qin = q0 + lane < P;
    int eq[4];
#pragma unroll
    for (int h = 0; h < 4; h++) {
        const int q = q0 + warp * 4 + h;
        eq[h] = q < P ? expo_q[p0 + q] : -10000;
    }
    uint8_t *base = slices + sl_off[b];
    for (int kc = 0; kc < G.n_kcN; kc++) {
#pragma unroll
        for (int h = 0; h < C / 8; h++) {
            const int i = kc * C + warp + 8 * h;
            t[lane][warp + 8 * h] = (i < N && qin) ? StageOf<V>::get(E[(int64_t)i * ld + q0 + lane]) : StageOf<V>::zero();
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const int ql = warp * 4 + h, q = q0 + ql;
            if (q >= G.P16) break;
            // lane L packs functions L, L + 32 (, L + 64, L + 96) of the chunk into its word: both
            // operands of the density's product (this A and slice_np_kernel's B) order K this way
            // inside each chunk, which leaves every slice product unchanged and reads the staging
            // rows without bank conflicts
            TT x[LC];
#pragma unroll
            for (int c = 0; c < LC; c++) x[c] = t[ql][lane + 32 * c];
            uint32_t wd[S];
            lane_digit_words<S, F>(x, eq[h], wd);
            const uint32_t off = tc::sw128_byte((uint32_t)q, (uint32_t)(4 * lane));
#pragma unroll
            for (int sl = 0; sl < S; sl++) *reinterpret_cast<uint32_t *>(base + G.nA_block(sl, kc) + off) = wd[sl];
        }
        __syncthreads();
    }
}

// P'_ij = c_IJ P[rel_i][rel_j] over TN-function tiles I = i/TN <= J = j/TN (c_II = 1,
// c_IJ = 2; every (i, j) with c = 1 when full), read from P's upper triangle, with the batch's
// exponent from slice_nphi_kernel. One CTA per (batch, 16 rows j), one warp per row, 2 or 4
// functions i per lane (i = lane + 32 c inside the chunk; one 128-byte row segment per slice).
template <int S, int F>
__global__ void __launch_bounds__(256) slice_np_kernel(DevSystem s, int32_t b0, uint8_t *__restrict__ slices,
                                                      const int64_t *__restrict__ sl_off,
                                                      const int32_t *__restrict__ expo_b,
                                                      const int32_t *__restrict__ tn_b, int full) {
    const int b = b0 + blockIdx.x, m = s.sys.bmol[b];
    const int P = s.batch_off[b + 1] - s.batch_off[b];
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    if (N == 0) return;
    constexpr int C = nao_chunk_cols(F), LC = C / 32;
    const SplitGeom G(P, N, S, 0, F);
    const int j0 = blockIdx.y * 16;
    if (j0 >= G.R16) return;
    const int32_t *rel = s.rel_idx + s.rel_off[b];
    const int TN = tn_b[b], e = expo_b[b];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *base = slices + sl_off[b];
#pragma unroll 1
    for (int h = 0; h < 2; h++) {
        const int j = j0 + warp * 2 + h;  // < R16: R16 is a multiple of 16
        const bool jin = j < N;
        const int64_t gj = jin ? rel[j] : 0;
        const int tj = tile_of(j, TN);
        for (int kc = 0; kc < G.n_kcN; kc++) {
            double xp[LC];
#pragma unroll
            for (int hh = 0; hh < LC; hh++) {
                const int i = C * kc + lane + 32 * hh;  // the K order of slice_nphi_kernel
                double x = 0.0;
                if (jin && i < N && (full || tile_of(i, TN) <= tj)) {
                    const int64_t gi = rel[i];
                    x = gi <= gj ? p_elem(s, m, gi, gj) : p_elem(s, m, gj, gi);
                    // c_IJ = 2 off the diagonal tiles: exact, as one more in the exponent field
                    // (zero and subnormal values, which give no digits, are left as they are)
                    const long long pb = __double_as_longlong(x);
                    if (!full && tile_of(i, TN) < tj && split_bits::biased_exponent(pb) != 0)
                        x = __longlong_as_double(pb + (1LL << 52));
                }
                xp[hh] = x;
            }
            uint32_t wd[S];
            lane_digit_words<S, F>(xp, e, wd);
            const uint32_t off = tc::sw128_byte((uint32_t)j, (uint32_t)(4 * lane));
#pragma unroll
            for (int sl = 0; sl < S; sl++) *reinterpret_cast<uint32_t *>(base + G.nB_block(S, sl, kc) + off) = wd[sl];
        }
    }
}

// ----------------------------------------------------------------------------------------
// Slice-product pipeline of the persistent contraction kernels. Shared memory: a ring of
// ring_slots(S) A-tile buffers (128 rows x 64 bf16, 16 KB, one slice of one K chunk each) and two sets of S
// B-tile buffers (TN rows, TN x 128 B). Producer (one lane): for each K chunk, the S B slices
// into B set kc % 2, then the S A slices one by one into the ring, each copy a single bulk
// (TMA) transfer completing on a "full" mbarrier. MMA issuer (one lane): for each A slice s,
// the pairs (s, t) with s + t < S as one 128 x TN(S-s) x 16 tcgen05.mma per K step (two where
// TN(S-s) > 256) into accumulator groups s .. S-1 (tensor-memory columns TN s ...); commits
// release A buffers and B sets back to the producer through "empty" mbarriers. The phases of
// the ring and of the B sets continue over all the accumulations a CTA runs. Every wait is
// bounded; on a timeout the CTA records NAO_ERR_TIMEOUT and skips the rest of its work.
// ----------------------------------------------------------------------------------------
constexpr int kMaxRing = 8;
constexpr size_t kSmemOptin = 232448;  // shared memory a CTA may opt into on this GPU (227 KB)
constexpr size_t kStaticSmem = 2048;   // room for the CTA's static shared memory (the PPipe barriers)

// A-ring slots: as many 16 KB A tiles as fit beside the two B sets (S tiles of TN rows each),
// at most kMaxRing: 8 for 11-12 bf16 slices (TN = 32), 6 for 10 (TN = 48), 7 for 14 e4m3 slices.
// A deeper ring lets the producer's copies run further ahead of the MMAs that wait for them.
__host__ __device__ constexpr int ring_slots(int S, int F) {
    return (int)((kSmemOptin - kStaticSmem - 1024 - 2 * (size_t)S * nao_split_tn(S, F) * 128) / 16384) < kMaxRing
               ? (int)((kSmemOptin - kStaticSmem - 1024 - 2 * (size_t)S * nao_split_tn(S, F) * 128) / 16384)
               : kMaxRing;
}

__host__ __device__ constexpr size_t pipe_smem_bytes(int S, int F) {
    return (size_t)ring_slots(S, F) * 16384 + 2 * (size_t)S * nao_split_tn(S, F) * 128 + 1024;
}
static_assert(ring_slots(12, 0) >= 4 && ring_slots(10, 0) >= 4 && ring_slots(4, 0) >= 4 && ring_slots(16, 1) >= 4,
              "A ring too shallow");
static_assert(pipe_smem_bytes(12, 0) + kStaticSmem <= kSmemOptin && pipe_smem_bytes(10, 0) + kStaticSmem <= kSmemOptin &&
                  pipe_smem_bytes(16, 1) + kStaticSmem <= kSmemOptin,
              "split pipeline exceeds shared memory");

// Integer recombination of the S group accumulators M_g (|M_g| < 2^24, exact) for 16 columns of
// this thread's row, in units of 2^(e_i + e_j):
//   bf16 (base 64): hi = sum_{g<=6} M_g 64^(6-g) [units 2^-48], lo = sum_{7<=g<=9} M_g 64^(9-g)
//     [2^-66], lo2 = sum_{g>=10} M_g 64^(12-g) [2^-84] (S = 11, 12 only);
//   e4m3 (base 32): hi = sum_{g<=7} M_g 32^(7-g) [units 2^-45], lo = sum_{g>=8} M_g 32^(15-g)
//     [2^-85] (S <= 16); lo2 stays 0.
// Every part is exact in 64 bits (below 2^60.1).
struct Parts16 {
    long long hi[16], lo[16], lo2[16];
};

template <int TN, int F>
__device__ __forceinline__ void combine16(uint32_t tm_row, int c0, int S, Parts16 &v) {
    constexpr int B = nao_digit_bits(F), GH = F == NAO_DIGITS_E4M3 ? 7 : 6, GL = F == NAO_DIGITS_E4M3 ? 15 : 9;
#pragma unroll
    for (int jj = 0; jj < 16; jj++) v.hi[jj] = v.lo[jj] = v.lo2[jj] = 0;
    // three groups' loads in flight per wait
    for (int g0 = 0; g0 < S; g0 += 3) {
        uint32_t r[3][16];
#pragma unroll
        for (int d = 0; d < 3; d++)
            if (g0 + d < S) tc::tmem_ld16(tm_row + (uint32_t)((g0 + d) * TN + c0), r[d]);
        tc::tmem_ld_wait();
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const int g = g0 + d;
            if (g >= S) break;
            const int part = g <= GH ? 0 : (g <= GL ? 1 : 2);
            const long long w = 1LL << (B * (part == 0 ? GH - g : (part == 1 ? GL - g : 12 - g)));
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const long long m = (long long)__float2int_rn(__uint_as_float(r[d][jj]));
                if (part == 0) v.hi[jj] += m * w;
                else if (part == 1) v.lo[jj] += m * w;
                else v.lo2[jj] += m * w;
            }
        }
    }
}

// An H element from its parts as one 64-bit integer v and a tier t, the value being
// v 2^(e_i + e_j - h_unit<F>(t)):
//   bf16: lo' = lo + round(lo2 / 2^18); t = 0 (|hi| < 2^44): hi 2^18 + lo' exactly (unit 66);
//         t = 1: 4 hi + round(lo' / 2^16) (unit 50; |4 hi| >= 2^46, relative error <= 2^-47);
//   e4m3: t = 0 (|hi| < 2^22): hi 2^40 + lo exactly (unit 85); t = 1 (|hi| < 2^40):
//         hi 2^22 + round(lo / 2^18) (unit 67; relative error <= 2^-45); t = 2:
//         4 hi + round(lo / 2^38) (unit 47; relative error <= 2^-43).
// (hi is in units of 2^-45 and lo of 2^-85 throughout: hi 2^k in units of 2^-(45 + k).)
template <int F>
__device__ __forceinline__ long long h_int(long long hi, long long lo, long long lo2, int &t) {
    if constexpr (F == NAO_DIGITS_BF16) {
        const long long l = lo + ((lo2 + (1LL << 17)) >> 18);
        if (hi > -(1LL << 44) && hi < (1LL << 44)) {
            t = 0;
            return (hi << 18) + l;
        }
        t = 1;
        return (hi << 2) + ((l + (1LL << 15)) >> 16);
    } else {
        if (hi > -(1LL << 22) && hi < (1LL << 22)) {
            t = 0;
            return (hi << 40) + lo;
        }
        if (hi > -(1LL << 40) && hi < (1LL << 40)) {
            t = 1;
            return (hi << 22) + ((lo + (1LL << 17)) >> 18);
        }
        t = 2;
        return (hi << 2) + ((lo + (1LL << 37)) >> 38);
    }
}
template <int F>
__device__ __forceinline__ int h_unit(int t) {
    return F == NAO_DIGITS_BF16 ? (t == 0 ? 66 : 50) : (t == 0 ? 85 : (t == 1 ? 67 : 47));
}
// A density T element as one 64-bit integer in units of 2^(e_q + e_b - n_unit<F>): 4 hi +
// round(lo' / 2^16) (bf16, unit 50) or 4 hi + round(lo / 2^38) (e4m3, unit 47); |4 hi| < 2^62.1,
// rounded by at most half a unit.
template <int F>
__device__ __forceinline__ long long n_int(long long hi, long long lo, long long lo2) {
    if constexpr (F == NAO_DIGITS_BF16) {
        const long long l = lo + ((lo2 + (1LL << 17)) >> 18);
        return (hi << 2) + ((l + (1LL << 15)) >> 16);
    } else {
        return (hi << 2) + ((lo + (1LL << 37)) >> 38);
    }
}
template <int F>
__host__ __device__ constexpr int n_unit() { return F == NAO_DIGITS_BF16 ? 50 : 47; }

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

// Persistent, warp-specialised H contraction: one CTA per SM walks the work items w =
// blockIdx.x, blockIdx.x + gridDim.x, ... Warp 4 (lane 0) loads the operands into the A ring and
// the two B sets, its phases continuing over all items; warp 5 (lane 0) issues the MMAs of one
// item after the other into the single accumulator set; warps 0-3 (128 threads, one accumulator
// row each) read an item's accumulators into registers, hand tensor memory back to the MMA warp
// ("acc_empty") and then scatter into H while the next item's MMAs run, so the scatter, the
// tensor-memory reads and the next item's first loads overlap the MMAs.
// The B tiles t = 0 .. nb-1 of one A slice as MMA pieces: one piece of nb TN columns up to
// N = 256, else two halves of ceil(nb / 2) and floor(nb / 2) tiles (each at most 256 columns,
// since nb TN <= 512, the tensor memory of one accumulator set). Every piece starts on a whole
// tile, so on a multiple of 8 rows (one 128-byte swizzle atom). Two halves, issued alternately,
// write disjoint accumulator columns: an MMA that accumulates into the columns of the one just
// issued waits for it (about 97 cycles at this size, against about 60 for other columns), and
// equal halves leave no narrow piece whose fixed cost exceeds its work.
struct MmaPieces {
    int n, c0[2], cols[2];
    __device__ __forceinline__ MmaPieces(int nb, int TN) {
        if (nb * TN <= 256) {
            n = 1;
            c0[0] = 0;
            cols[0] = nb * TN;
            c0[1] = cols[1] = 0;
        } else {
            const int h = (nb + 1) / 2;
            n = 2;
            c0[0] = 0;
            cols[0] = h * TN;
            c0[1] = h * TN;
            cols[1] = (nb - h) * TN;
        }
    }
};

struct PPipe {
    uint64_t fullA[kMaxRing], emptyA[kMaxRing], fullB[2], emptyB[2];
    uint64_t acc_full, acc_empty, fin;
    uint32_t tmem;
    int abort;
};

struct HItem {  // geometry of one H work item
    const uint8_t *a0, *b0;
    size_t blk;
    uint32_t a_bytes, b_bytes;
    int n_kc, kc0, kc1, neg16, b, m, N, ti, tj;  // K chunks [kc0, kc1) of the item's segment
};

template <int TN, int F>
__device__ __forceinline__ HItem h_item(const DevSystem &s, const HWork *work, int32_t w, const uint8_t *slices,
                                        const int64_t *sl_off, const int32_t *neg16, int S) {
    HItem h;
    const HWork it = work[w];
    h.b = it.batch;
    h.ti = it.ti;
    h.tj = it.tj;
    h.m = s.sys.bmol[h.b];
    const int P = s.batch_off[h.b + 1] - s.batch_off[h.b];
    h.N = s.rel_off[h.b + 1] - s.rel_off[h.b];
    const SplitGeom G(P, h.N, S, TN, F);
    const uint8_t *base = slices + sl_off[h.b];
    h.blk = (size_t)G.R16 * 128;
    h.a0 = base + (size_t)it.ti * 128 * 128;
    h.b0 = base + (size_t)it.tj * TN * 128;
    h.a_bytes = (uint32_t)min(128, G.R16 - it.ti * 128) * 128u;
    h.b_bytes = (uint32_t)min(TN, G.R16 - it.tj * TN) * 128u;
    h.n_kc = G.n_kc;
    nao_split_h_seg_range(G.n_kc, nao_split_h_nseg(P, S, F), it.pad, S, h.kc0, h.kc1, F);
    h.neg16 = neg16[h.b];
    return h;
}

template <int TN, int F>
__global__ void __launch_bounds__(192, 1)
    h_tc_kernel(DevSystem s, const HWork *__restrict__ work, int32_t w0, int32_t n_work, const uint8_t *__restrict__ slices,
                const int64_t *__restrict__ sl_off, const int32_t *__restrict__ expo,
                const int32_t *__restrict__ neg16, int S, int scatter, int32_t *__restrict__ err) {
    constexpr uint32_t B_BLOCK = TN * 128;
    extern __shared__ uint8_t smem_dyn[];
    __shared__ PPipe pp;
    uint8_t *smem = align1024(smem_dyn);
    const int RING = ring_slots(S, F);
    uint8_t *sA = smem, *sB = smem + (size_t)RING * 16384;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING; i++) {
            tc::mbar_init(&pp.fullA[i], 1);
            tc::mbar_init(&pp.emptyA[i], 1);
        }
        for (int i = 0; i < 2; i++) {
            tc::mbar_init(&pp.fullB[i], 1);
            tc::mbar_init(&pp.emptyB[i], 1);
        }
        tc::mbar_init(&pp.acc_full, 1);
        tc::mbar_init(&pp.acc_empty, 4);  // one arrival per accumulator-reading warp
        tc::mbar_init(&pp.fin, 1);
        tc::fence_mbar_init();
        pp.abort = *(volatile int32_t *)err != 0 ? 1 : 0;  // a timeout earlier in this launch
    }
    __syncwarp();
    if (warp == 0) {
        tc::tmem_alloc(&pp.tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = pp.tmem;
    volatile int *abort = &pp.abort;

    if (warp == 4) {
        // ---- producer ----
        if (lane == 0) {
            int gk = 0;
            for (int w = blockIdx.x; w < n_work && !*abort; w += gridDim.x) {
                const HItem h = h_item<TN, F>(s, work, w0 + w, slices, sl_off, neg16, S);
                const bool more = w + (int)gridDim.x < n_work;
                HItem hn = h;
                if (more) hn = h_item<TN, F>(s, work, w0 + w + gridDim.x, slices, sl_off, neg16, S);
                for (int kc = h.kc0; kc < h.kc1; kc++, gk++) {
                    // the next K chunk's slices (or the next item's first) towards L2, so that the
                    // ring's copies come from L2
                    if (kc + 1 < h.kc1 || more) {
                        const HItem &hp = kc + 1 < h.kc1 ? h : hn;
                        const int kp = kc + 1 < h.kc1 ? kc + 1 : hn.kc0;
                        for (int t = 0; t < S; t++) {
                            tc::bulk_prefetch_l2(hp.b0 + ((size_t)t * hp.n_kc + kp) * hp.blk, hp.b_bytes);
                            tc::bulk_prefetch_l2(hp.a0 + ((size_t)t * hp.n_kc + kp) * hp.blk, hp.a_bytes);
                        }
                    }
                    const int bb = gk & 1, ub = gk >> 1;
                    if (ub >= 1 && !tc::mbar_wait(&pp.emptyB[bb], (ub - 1) & 1, kWaitCycles)) { *abort = 1; break; }
                    tc::mbar_arrive_expect_tx(&pp.fullB[bb], (uint32_t)S * h.b_bytes);
                    for (int t = 0; t < S; t++)
                        tc::bulk_g2s(sB + ((size_t)bb * S + t) * B_BLOCK, h.b0 + ((size_t)t * h.n_kc + kc) * h.blk,
                                     h.b_bytes, &pp.fullB[bb]);
                    for (int sa = 0; sa < S; sa++) {
                        const int idx = gk * S + sa, a = idx % RING, ua = idx / RING;
                        if (ua >= 1 && !tc::mbar_wait(&pp.emptyA[a], (ua - 1) & 1, kWaitCycles)) { *abort = 1; break; }
                        tc::mbar_arrive_expect_tx(&pp.fullA[a], h.a_bytes);
                        tc::bulk_g2s(sA + (size_t)a * 16384, h.a0 + ((size_t)sa * h.n_kc + kc) * h.blk, h.a_bytes,
                                     &pp.fullA[a]);
                    }
                    if (*abort) break;
                }
            }
        }
    } else if (warp == 5) {
        // ---- MMA issuer ----
        if (lane == 0) {
            int gk = 0, t = 0;
            for (int w = blockIdx.x; w < n_work && !*abort; w += gridDim.x, t++) {
                const HItem h = h_item<TN, F>(s, work, w0 + w, slices, sl_off, neg16, S);
                // the accumulators of the previous item have been read
                if (t >= 1 && !tc::mbar_wait(&pp.acc_empty, (t - 1) & 1, kWaitCycles)) { *abort = 1; break; }
                tc::fence_after_sync();
                for (int kc = h.kc0; kc < h.kc1 && !*abort; kc++, gk++) {
                    const int bb = gk & 1, ub = gk >> 1;
                    if (!tc::mbar_wait(&pp.fullB[bb], ub & 1, kWaitCycles)) { *abort = 1; break; }
                    const uint8_t *bset = sB + (size_t)bb * S * B_BLOCK;
                    const int first = kc == h.kc0 ? 0 : 1;  // the segment's first chunk overwrites the accumulators
                    for (int sa = 0; sa < S; sa++) {
                        const int idx = gk * S + sa, a = idx % RING, ua = idx / RING;
                        if (!tc::mbar_wait(&pp.fullA[a], ua & 1, kWaitCycles)) { *abort = 1; break; }
                        tc::fence_after_sync();
                        const uint64_t ad = tc::sdesc_sw128(tc::smem_addr(sA + (size_t)a * 16384));
                        // pairs (sa, t = 0 .. S-1-sa): one MMA per K step over the S - sa B tiles,
                        // or two halves of them above N = 256 (mma_pieces), issued K step by K
                        // step so that consecutive MMAs alternate between the halves' columns
                        const MmaPieces pc(S - sa, TN);
#pragma unroll
                        for (int ks = 0; ks < 4; ks++) {
                            const bool neg = kc * 4 + ks < h.neg16;
                            const uint32_t acc = (first | sa | ks) ? 1u : 0u;
                            for (int p = 0; p < pc.n; p++) {
                                const uint32_t idesc = tc::idesc_digits<F>(128, pc.cols[p]);
                                const uint64_t bd = tc::sdesc_sw128(tc::smem_addr(bset + (size_t)pc.c0[p] * 128));
                                tc::mma_digits<F>(tm + (uint32_t)(sa * TN + pc.c0[p]), ad + 2 * ks, bd + 2 * ks,
                                                  neg ? (idesc | (1u << 14)) : idesc, acc);
                            }
                        }
                        tc::mma_commit(&pp.emptyA[a]);
                    }
                    tc::mma_commit(&pp.emptyB[bb]);
                }
                if (*abort) break;
                tc::mma_commit(&pp.acc_full);  // this item's accumulators are complete
            }
            // every issued MMA has completed before tensor memory is released
            tc::mma_commit(&pp.fin);
            if (!tc::mbar_wait(&pp.fin, 0, kWaitCycles)) *abort = 1;
        }
    } else {
        // ---- accumulator readers and scatter (warps 0-3) ----
        int t = 0;
        const uint32_t tm_row = tm + ((uint32_t)(warp * 32) << 16);
        for (int w = blockIdx.x; w < n_work; w += gridDim.x, t++) {
            const HItem h = h_item<TN, F>(s, work, w0 + w, slices, sl_off, neg16, S);
            if (*abort || !tc::mbar_wait(&pp.acc_full, t & 1, kWaitCycles)) { *abort = 1; break; }
            tc::fence_after_sync();
            const int i = h.ti * 128 + warp * 32 + lane;
            const bool row_ok = i < h.N;
            const int32_t *rel = s.rel_idx + s.rel_off[h.b];
            const int32_t *ex = expo + s.rel_off[h.b];
            const int ei = row_ok ? ex[i] : -10000;
            // h_ij as one 64-bit integer v and a tier t (h_int: exact where the high part is
            // small, else relative error <= 2^-43), formed before tensor memory is handed back;
            // the conversion and the product by 2^(e_i + e_j - h_unit(t)) after.
            long long val[TN];
            uint64_t t1_mask = 0, t2_mask = 0;
#pragma unroll
            for (int c0 = 0; c0 < TN; c0 += 16) {
                Parts16 v;
                combine16<TN, F>(tm_row, c0, S, v);
#pragma unroll
                for (int jj = 0; jj < 16; jj++) {
                    int t;
                    val[c0 + jj] = h_int<F>(v.hi[jj], v.lo[jj], v.lo2[jj], t);
                    t1_mask |= (uint64_t)(t == 1) << (c0 + jj);
                    t2_mask |= (uint64_t)(t == 2) << (c0 + jj);
                }
            }
            // tensor memory is free for the next item
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&pp.acc_empty);
            if (scatter && row_ok) {
                const int64_t gi = rel[i];
#pragma unroll
                for (int jj = 0; jj < TN; jj++) {
                    const int j = h.tj * TN + jj;
                    if (j < h.N && j >= i) {
                        const int ej = ex[j];
                        const int t = ((t1_mask >> jj) & 1) ? 1 : (((t2_mask >> jj) & 1) ? 2 : 0);
                        const double x = (ei > -10000 && ej > -10000) ? (double)val[jj] * pow2(ei + ej - h_unit<F>(t)) : 0.0;
                        h_add(s, h.m, gi, rel[j], x);
                    }
                }
            }
        }
    }
    if (*abort && threadIdx.x == 0) atomicExch(err, (int)NAO_ERR_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tm, 512);
}

// Density contraction, persistent and warp-specialised as h_tc_kernel: one CTA per SM walks
// the work items (batch, 128-point tile, nJ TN-function tiles) w = blockIdx.x, blockIdx.x +
// gridDim.x, ...; each item is nJ accumulations T_qJ = Phi_q P'_J (K = the functions up to
// tile J, where P' is nonzero), one after another through the single accumulator set. Warps
// 0-3 (one point each) read tile J's accumulators, hand tensor memory back and then add
// sum_j T_qj phi_qj to the point's n in registers while tile J+1's MMAs run; after the last
// tile they store n (no atomics: one item owns each point).
// GRADN (density gradient, Sec. 2): P' = P over all of K, and the epilogue also forms
// grad n_q = 2 sum_j T_qj grad phi_qj from the rows [phi | grad phi] of 4 Ppad.
struct NItem {  // geometry of one density work item
    const uint8_t *a0, *b0;  // A: slice 0, chunk 0 of the point tile; B: slice 0, chunk 0, tile 0
    size_t a_s, a_kc, b_s, b_kc;
    uint32_t a_bytes;
    int nJ, n_kcN, R16, b, m, p0, P, Ppad, N, ti;
};

template <int TN, int F>
__device__ __forceinline__ NItem n_item(const DevSystem &s, const HWork *work, int32_t w, const uint8_t *slices,
                                        const int64_t *sl_off, int S) {
    NItem h;
    const HWork it = work[w];  // batch, 128-point tile, number of TN-function tiles
    h.b = it.batch;
    h.ti = it.ti;
    h.nJ = it.tj;
    h.m = s.sys.bmol[h.b];
    h.p0 = s.batch_off[h.b];
    h.P = s.batch_off[h.b + 1] - h.p0;
    h.Ppad = (h.P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    h.N = s.rel_off[h.b + 1] - s.rel_off[h.b];
    const SplitGeom G(h.P, h.N, S, TN, F);
    const uint8_t *base = slices + sl_off[h.b];
    h.a0 = base + G.nA_block(0, 0) + (size_t)it.ti * 128 * 128;
    h.a_s = (size_t)G.n_kcN * G.P16 * 128;
    h.a_kc = (size_t)G.P16 * 128;
    h.b0 = base + G.nB_block(S, 0, 0);
    h.b_s = (size_t)G.n_kcN * G.R16 * 128;
    h.b_kc = (size_t)G.R16 * 128;
    h.a_bytes = (uint32_t)min(128, G.P16 - it.ti * 128) * 128u;
    h.n_kcN = G.n_kcN;
    h.R16 = G.R16;
    return h;
}

// K chunks of tile J: P' is zero for basis functions beyond tile J, so K stops at TN (J + 1)
// (all of K for GRADN)
template <int TN, bool GRADN, int F>
__device__ __forceinline__ int n_item_kc(const NItem &h, int J) {
    constexpr int C = nao_chunk_cols(F);
    const int nk = GRADN ? h.n_kcN : ((J + 1) * TN + C - 1) / C;
    return nk < h.n_kcN ? nk : h.n_kcN;
}

// MODE 0: n; 1: n and grad n (GRADN); 2: the density Hessian's first pass (A = Phi: n, grad n and
// 2 sum_j T_qj d_a d_b phi_qj into hess); 3: a later pass (A = d_hc Phi: hess_(hc, b) +=
// 2 sum_j T_qj d_b phi_qj for b >= hc). Modes 0, 1 read the float-float evaluation at scr_off,
// modes 2, 3 the Hessian's 10-row FP64 evaluation at eoff.
template <int TN, int MODE, int F>
__global__ void __launch_bounds__(192, 1)
    n_tc_kernel(DevSystem s, const HWork *__restrict__ work, int32_t w0, int32_t n_work, const uint8_t *__restrict__ slices,
                const int64_t *__restrict__ sl_off, const int32_t *__restrict__ expo_q,
                const int32_t *__restrict__ expo_b, const void *__restrict__ scratch_v,
                const int64_t *__restrict__ eoff, int S, int hc, double *__restrict__ hess,
                int32_t *__restrict__ err) {
    constexpr bool GRADN = MODE >= 1;  // P' over all of K
    using V = typename std::conditional<(MODE >= 2), double, FF2>::type;
    const V *scratch = static_cast<const V *>(scratch_v);
    constexpr uint32_t B_BLOCK = TN * 128;
    extern __shared__ uint8_t smem_dyn[];
    __shared__ PPipe pp;
    uint8_t *smem = align1024(smem_dyn);
    const int RING = ring_slots(S, F);
    uint8_t *sA = smem, *sB = smem + (size_t)RING * 16384;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING; i++) {
            tc::mbar_init(&pp.fullA[i], 1);
            tc::mbar_init(&pp.emptyA[i], 1);
        }
        for (int i = 0; i < 2; i++) {
            tc::mbar_init(&pp.fullB[i], 1);
            tc::mbar_init(&pp.emptyB[i], 1);
        }
        tc::mbar_init(&pp.acc_full, 1);
        tc::mbar_init(&pp.acc_empty, 4);  // one arrival per accumulator-reading warp
        tc::mbar_init(&pp.fin, 1);
        tc::fence_mbar_init();
        pp.abort = *(volatile int32_t *)err != 0 ? 1 : 0;  // a timeout earlier in this launch
    }
    __syncwarp();
    if (warp == 0) {
        tc::tmem_alloc(&pp.tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = pp.tmem;
    volatile int *abort = &pp.abort;

    if (warp == 4) {
        // ---- producer ----
        if (lane == 0) {
            int gk = 0;
            for (int w = blockIdx.x; w < n_work && !*abort; w += gridDim.x) {
                const NItem h = n_item<TN, F>(s, work, w0 + w, slices, sl_off, S);
                for (int J = 0; J < h.nJ && !*abort; J++) {
                    const int nk = n_item_kc<TN, (MODE >= 1), F>(h, J);
                    const uint8_t *bJ = h.b0 + (size_t)J * TN * 128;
                    const uint32_t b_bytes = (uint32_t)min(TN, h.R16 - J * TN) * 128u;
                    for (int kc = 0; kc < nk; kc++, gk++) {
                        // the next K chunk of this tile (or the next tile's first) towards L2
                        {
                            const bool same = kc + 1 < nk;
                            const int Jp = same ? J : J + 1, kp = same ? kc + 1 : 0;
                            if (Jp < h.nJ) {
                                const uint8_t *bp = h.b0 + (size_t)Jp * TN * 128;
                                const uint32_t bpb = (uint32_t)min(TN, h.R16 - Jp * TN) * 128u;
                                for (int t = 0; t < S; t++) {
                                    tc::bulk_prefetch_l2(bp + t * h.b_s + kp * h.b_kc, bpb);
                                    tc::bulk_prefetch_l2(h.a0 + t * h.a_s + kp * h.a_kc, h.a_bytes);
                                }
                            }
                        }
                        const int bb = gk & 1, ub = gk >> 1;
                        if (ub >= 1 && !tc::mbar_wait(&pp.emptyB[bb], (ub - 1) & 1, kWaitCycles)) { *abort = 1; break; }
                        tc::mbar_arrive_expect_tx(&pp.fullB[bb], (uint32_t)S * b_bytes);
                        for (int t = 0; t < S; t++)
                            tc::bulk_g2s(sB + ((size_t)bb * S + t) * B_BLOCK, bJ + t * h.b_s + kc * h.b_kc, b_bytes,
                                         &pp.fullB[bb]);
                        for (int sa = 0; sa < S; sa++) {
                            const int idx = gk * S + sa, a = idx % RING, ua = idx / RING;
                            if (ua >= 1 && !tc::mbar_wait(&pp.emptyA[a], (ua - 1) & 1, kWaitCycles)) { *abort = 1; break; }
                            tc::mbar_arrive_expect_tx(&pp.fullA[a], h.a_bytes);
                            tc::bulk_g2s(sA + (size_t)a * 16384, h.a0 + sa * h.a_s + kc * h.a_kc, h.a_bytes, &pp.fullA[a]);
                        }
                        if (*abort) break;
                    }
                }
            }
        }
    } else if (warp == 5) {
        // ---- MMA issuer ----
        if (lane == 0) {
            int gk = 0, t = 0;
            for (int w = blockIdx.x; w < n_work && !*abort; w += gridDim.x) {
                const NItem h = n_item<TN, F>(s, work, w0 + w, slices, sl_off, S);
                for (int J = 0; J < h.nJ && !*abort; J++, t++) {
                    const int nk = n_item_kc<TN, (MODE >= 1), F>(h, J);
                    // the accumulators of the previous tile have been read
                    if (t >= 1 && !tc::mbar_wait(&pp.acc_empty, (t - 1) & 1, kWaitCycles)) { *abort = 1; break; }
                    tc::fence_after_sync();
                    for (int kc = 0; kc < nk && !*abort; kc++, gk++) {
                        const int bb = gk & 1, ub = gk >> 1;
                        if (!tc::mbar_wait(&pp.fullB[bb], ub & 1, kWaitCycles)) { *abort = 1; break; }
                        const uint8_t *bset = sB + (size_t)bb * S * B_BLOCK;
                        for (int sa = 0; sa < S; sa++) {
                            const int idx = gk * S + sa, a = idx % RING, ua = idx / RING;
                            if (!tc::mbar_wait(&pp.fullA[a], ua & 1, kWaitCycles)) { *abort = 1; break; }
                            tc::fence_after_sync();
                            const uint64_t ad = tc::sdesc_sw128(tc::smem_addr(sA + (size_t)a * 16384));
                            // pairs (sa, t = 0 .. S-1-sa), issued as in h_tc_kernel
                            const MmaPieces pc(S - sa, TN);
#pragma unroll
                            for (int ks = 0; ks < 4; ks++) {
                                const uint32_t acc = (kc | sa | ks) ? 1u : 0u;
                                for (int p = 0; p < pc.n; p++) {
                                    const uint32_t idesc = tc::idesc_digits<F>(128, pc.cols[p]);
                                    const uint64_t bd = tc::sdesc_sw128(tc::smem_addr(bset + (size_t)pc.c0[p] * 128));
                                    tc::mma_digits<F>(tm + (uint32_t)(sa * TN + pc.c0[p]), ad + 2 * ks, bd + 2 * ks, idesc,
                                                      acc);
                                }
                            }
                            tc::mma_commit(&pp.emptyA[a]);
                        }
                        tc::mma_commit(&pp.emptyB[bb]);
                    }
                    if (*abort) break;
                    tc::mma_commit(&pp.acc_full);  // tile J's accumulators are complete
                }
            }
            // every issued MMA has completed before tensor memory is released
            tc::mma_commit(&pp.fin);
            if (!tc::mbar_wait(&pp.fin, 0, kWaitCycles)) *abort = 1;
        }
    } else {
        // ---- accumulator readers and the n epilogue (warps 0-3) ----
        int t = 0;
        const uint32_t tm_row = tm + ((uint32_t)(warp * 32) << 16);
        for (int w = blockIdx.x; w < n_work && !*abort; w += gridDim.x) {
            const NItem h = n_item<TN, F>(s, work, w0 + w, slices, sl_off, S);
            const int q = h.ti * 128 + warp * 32 + lane;
            const bool row_ok = q < h.P;
            const V *E = scratch + eoff[h.b];
            const int64_t ld = MODE >= 2 ? 10 * (int64_t)h.Ppad : (GRADN ? 4 * (int64_t)h.Ppad : (int64_t)h.Ppad);
            // sum_j T_qj phi_qj (and grad phi) in units of 2^(e_q + e_b - n_unit): each T_qj as one
            // 64-bit integer in those units (n_int: 2^-50 with bf16 digits, 2^-47 with e4m3),
            // rounded by at most half a unit: about the split's own truncation at 10 bf16 slices
            // (the dropped groups g >= S reach K (S + 1) 2^(e_q + e_b - 6S - 2)) and below the FP64
            // evaluation's rounding in n. Then one conversion and one FMA per product, all integer
            // work done before tensor memory is handed back (no FP64 arithmetic on that path).
            double part = 0.0, gpart[3] = {0.0, 0.0, 0.0}, hpart[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int J = 0; J < h.nJ; J++, t++) {
                if (*abort || !tc::mbar_wait(&pp.acc_full, t & 1, kWaitCycles)) { *abort = 1; break; }
                tc::fence_after_sync();
                long long val[TN];
#pragma unroll
                for (int c0 = 0; c0 < TN; c0 += 16) {
                    Parts16 v;
                    combine16<TN, F>(tm_row, c0, S, v);
#pragma unroll
                    for (int jj = 0; jj < 16; jj++) val[c0 + jj] = n_int<F>(v.hi[jj], v.lo[jj], v.lo2[jj]);
                }
                // tensor memory is free for the next tile
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&pp.acc_empty);
                if (row_ok) {
                    // the next tile's rows of phi towards L2 while this tile's products run
                    if (J + 1 < h.nJ) {
                        const V *fn = E + (int64_t)(J + 1) * TN * ld + q;
                        const int jn1 = min(TN, h.N - (J + 1) * TN);
                        for (int jj = 0; jj < jn1; jj++) asm volatile("prefetch.global.L2 [%0];" ::"l"(fn + jj * ld));
                    }
                    const int jn = min(TN, h.N - J * TN);
                    const V *f = E + (int64_t)J * TN * ld + q;
#pragma unroll
                    for (int jj = 0; jj < TN; jj++) {
                        if (jj < jn) {
                            const double vj = (double)val[jj];
                            const V *fj = f + jj * ld;
                            if (MODE <= 2) part = fma(vj, double(fj[0]), part);
                            if (MODE == 1 || MODE == 2)
#pragma unroll
                                for (int d = 0; d < 3; d++) gpart[d] = fma(vj, double(fj[(d + 1) * h.Ppad]), gpart[d]);
                            if (MODE == 2)
#pragma unroll
                                for (int k = 0; k < 6; k++) hpart[k] = fma(vj, double(fj[(4 + k) * h.Ppad]), hpart[k]);
                            if (MODE == 3)  // T^hc_qj d_b phi_qj, b = 1..3 in hpart[b - 1]
#pragma unroll
                                for (int d = 0; d < 3; d++) hpart[d] = fma(vj, double(fj[(d + 1) * h.Ppad]), hpart[d]);
                        }
                    }
                }
            }
            if (*abort) break;
            if (row_ok) {
                const int eq = expo_q[h.p0 + q], eb = expo_b[h.b];
                const bool live = eq > -10000 && eb > -10000;
                const double sc = pow2(eq + eb - n_unit<F>());
                if (MODE <= 2) *n_at(s, h.m, h.p0 + q) = live ? part * sc : 0.0;
                if (MODE == 1 || MODE == 2)
#pragma unroll
                    for (int d = 0; d < 3; d++) *gn_at(s, h.m, h.p0 + q, d) = live ? 2.0 * gpart[d] * sc : 0.0;
                if (MODE >= 2) {
                    // hess: component-major (xx, xy, xz, yy, yz, zz), the system's original point order
                    const int64_t np = s.sys.np[h.m], o = s.perm[h.p0 + q] - s.sys.poff[h.m];
                    if (MODE == 2) {
#pragma unroll
                        for (int k = 0; k < 6; k++) hess[k * np + o] = live ? 2.0 * hpart[k] * sc : 0.0;
                    } else {
                        // pair (hc, b) of components 1..3 -> 0, 1, 2 (x.), 3, 4 (y.), 5 (zz)
                        const int kb = (hc - 1) * 3 - ((hc - 1) * (hc - 2)) / 2 - hc;
#pragma unroll
                        for (int d = 0; d < 3; d++)
                            if (d + 1 >= hc && live) hess[(kb + d + 1) * np + o] += 2.0 * hpart[d] * sc;
                    }
                }
            }
        }
    }
    if (*abort && threadIdx.x == 0) atomicExch(err, (int)NAO_ERR_TIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tm, 512);
}

// sum over each density tile of 64 points of w n (then the deterministic final reduction)
__global__ void __launch_bounds__(256) wn_partial_kernel(DevSystem s, const DWork *__restrict__ work, int32_t w0,
                                                        double *__restrict__ ne_part) {
    __shared__ double red[8];
    const DWork it = work[w0 + blockIdx.x];
    const int p0 = s.batch_off[it.batch], P = s.batch_off[it.batch + 1] - p0;
    const int q = it.tp * NAO_TILE + threadIdx.x;
    double wn = 0.0;
    if (threadIdx.x < NAO_TILE && q < P) wn = s.pw[p0 + q] * *n_at(s, s.sys.bmol[it.batch], p0 + q);
    for (int o = 16; o > 0; o >>= 1) wn += __shfl_xor_sync(0xffffffffu, wn, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = wn;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += red[w];
        ne_part[w0 + blockIdx.x] = t;
    }
}

// The timeout path of the bounded waits, exercised without a stuck pipeline: one thread waits on
// an mbarrier that expects one arrival which never comes (no copy or MMA is in flight, so giving
// up leaves nothing behind), then records the timeout the way the contraction kernels do.
__global__ void wait_timeout_probe_kernel(long long max_cycles, int32_t *__restrict__ err) {
    __shared__ uint64_t bar;
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    if (!tc::mbar_wait(&bar, 0, max_cycles)) {
        atomicExch(err + 1, 1);
        atomicExch(err, (int)NAO_ERR_TIMEOUT);
    }
}

// Point exponents of the Hessian's four A operands (phi and the three gradient components, rows
// c = 0..3 of the 10-row FP64 evaluation): expo4[c n_points + batch_off[b] + q] from the binade
// of max_i |row c of function i at point q|. One CTA per batch.
__global__ void __launch_bounds__(256) hess_point_expo_kernel(DevSystem s, int32_t b0, const double *__restrict__ scratch,
                                                             const int64_t *__restrict__ hoff, int32_t *__restrict__ expo4,
                                                             int64_t n_points) {
    const int b = b0 + blockIdx.x;
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const double *E = scratch + hoff[b];
    const int64_t ld = 10 * (int64_t)Ppad;
    for (int idx = threadIdx.x; idx < 4 * P; idx += blockDim.x) {
        const int c = idx / P, q = idx - c * P;
        int mx = 0;
        for (int i = 0; i < N; i++) mx = max(mx, split_bits::biased_exponent(abs_bits(E[i * ld + (int64_t)c * Ppad + q])));
        expo4[c * n_points + p0 + q] = split_bits::exponent_of_binade(mx);
    }
}

}  // namespace

size_t split_smem_bytes(int S, int F) { return pipe_smem_bytes(S, F); }

cudaError_t launch_wait_timeout_probe(long long max_cycles, int32_t *err, cudaStream_t st) {
    wait_timeout_probe_kernel<<<1, 1, 0, st>>>(max_cycles, err);
    return cudaGetLastError();
}

// SMs of the current device (the persistent kernels' grid size).
static int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n <= 0)
        return 1;
    return n;
}

cudaError_t split_configure() {
    size_t bytes = 0;
    for (int S = 4; S <= NAO_SPLIT_MAX_SLICES; S++) bytes = std::max(bytes, split_smem_bytes(S, NAO_DIGITS_BF16));
    for (int S = 8; S <= NAO_SPLIT_MAX_SLICES_E4M3; S++) bytes = std::max(bytes, split_smem_bytes(S, NAO_DIGITS_E4M3));
    const void *fns[] = {(const void *)h_tc_kernel<48, 0>,    (const void *)h_tc_kernel<32, 0>,
                         (const void *)h_tc_kernel<32, 1>,    (const void *)n_tc_kernel<48, 0, 0>,
                         (const void *)n_tc_kernel<48, 1, 0>, (const void *)n_tc_kernel<48, 2, 0>,
                         (const void *)n_tc_kernel<48, 3, 0>, (const void *)n_tc_kernel<32, 0, 0>,
                         (const void *)n_tc_kernel<32, 1, 0>, (const void *)n_tc_kernel<32, 2, 0>,
                         (const void *)n_tc_kernel<32, 3, 0>, (const void *)n_tc_kernel<32, 0, 1>,
                         (const void *)n_tc_kernel<32, 1, 1>, (const void *)n_tc_kernel<32, 2, 1>,
                         (const void *)n_tc_kernel<32, 3, 1>};
    for (const void *f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Slice counts with compiled slicers: 4..12 with bf16 digits, 8..16 with e4m3 digits.
#define NAO_SPLIT_DISPATCH(S, F, CALL)                                                                 \
    if (F == NAO_DIGITS_E4M3) {                                                                        \
        switch (S) {                                                                                   \
            case 8: CALL(8, 1); break;                                                                 \
            case 9: CALL(9, 1); break;                                                                 \
            case 10: CALL(10, 1); break;                                                               \
            case 11: CALL(11, 1); break;                                                               \
            case 12: CALL(12, 1); break;                                                               \
            case 13: CALL(13, 1); break;                                                               \
            case 14: CALL(14, 1); break;                                                               \
            case 15: CALL(15, 1); break;                                                               \
            default: CALL(16, 1); break;                                                               \
        }                                                                                              \
    } else {                                                                                           \
        switch (S) {                                                                                   \
            case 4: CALL(4, 0); break;                                                                 \
            case 5: CALL(5, 0); break;                                                                 \
            case 6: CALL(6, 0); break;                                                                 \
            case 7: CALL(7, 0); break;                                                                 \
            case 8: CALL(8, 0); break;                                                                 \
            case 9: CALL(9, 0); break;                                                                 \
            case 10: CALL(10, 0); break;                                                               \
            case 11: CALL(11, 0); break;                                                               \
            default: CALL(12, 0); break;                                                               \
        }                                                                                              \
    }

cudaError_t launch_slice_h(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_rt, const double *scratch, uint32_t terms, uint8_t *slices, const int64_t *sl_off, int32_t *expo,
                           int32_t *neg16, int S, int F, cudaStream_t st) {
    if (b1 <= b0 || max_rt <= 0) return cudaSuccess;
    const FF2 *ev = reinterpret_cast<const FF2 *>(scratch);  // the split path's evaluation: float-float values
#define NAO_SLICE_H(SS, FF) \
    slice_h_kernel<SS, FF><<<dim3(b1 - b0, max_rt), 256, 0, st>>>(s, b0, ev, terms, slices, sl_off, expo, neg16)
    NAO_SPLIT_DISPATCH(S, F, NAO_SLICE_H)
#undef NAO_SLICE_H
    return cudaGetLastError();
}

cudaError_t launch_h_tc(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                        const int64_t *sl_off, const int32_t *expo, const int32_t *neg16, int S, int F, int tn,
                        int scatter, int32_t *err, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    const int grid = n_work < sm_count() ? n_work : sm_count();  // persistent: one CTA per SM
    const size_t sm = split_smem_bytes(S, F);
    if (F == NAO_DIGITS_E4M3 && tn == 32)
        h_tc_kernel<32, 1><<<grid, 192, sm, st>>>(s, work, w0, n_work, slices, sl_off, expo, neg16, S, scatter, err);
    else if (F == NAO_DIGITS_BF16 && tn == 48 && S <= 10)
        h_tc_kernel<48, 0><<<grid, 192, sm, st>>>(s, work, w0, n_work, slices, sl_off, expo, neg16, S, scatter, err);
    else if (F == NAO_DIGITS_BF16 && tn == 32)
        h_tc_kernel<32, 0><<<grid, 192, sm, st>>>(s, work, w0, n_work, slices, sl_off, expo, neg16, S, scatter, err);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_slice_n(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_qt, int32_t max_rt,
                           const double *scratch, uint8_t *slices, const int64_t *sl_off, const int32_t *expo_q,
                           int32_t *expo_b, const int32_t *tn_b, int S, int F, bool grad, cudaStream_t st) {
    if (b1 <= b0) return cudaSuccess;
    const FF2 *ev = reinterpret_cast<const FF2 *>(scratch);
    // y = 0: the exponent of P'; y >= 1: 32-point tiles (128 max_qt >= P16)
#define NAO_SLICE_NPHI(SS, FF)                                                                            \
    slice_nphi_kernel<SS, FF, FF2><<<dim3(b1 - b0, 4 * max_qt + 1), 256, 0, st>>>(                        \
        s, b0, ev, s.scr_off, 0, slices, sl_off, expo_q, expo_b, tn_b, grad ? 4 : 1, grad ? 1 : 0, 1)
    NAO_SPLIT_DISPATCH(S, F, NAO_SLICE_NPHI)
#undef NAO_SLICE_NPHI
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || max_rt <= 0) return e;
    // 16 rows per CTA (64 max_rt >= R16)
#define NAO_SLICE_NP(SS, FF) \
    slice_np_kernel<SS, FF><<<dim3(b1 - b0, 4 * max_rt), 256, 0, st>>>(s, b0, slices, sl_off, expo_b, tn_b, grad ? 1 : 0)
    NAO_SPLIT_DISPATCH(S, F, NAO_SLICE_NP)
#undef NAO_SLICE_NP
    return cudaGetLastError();
}

cudaError_t launch_slice_n_hess(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_qt, int32_t max_rt,
                                const double *scratch, const int64_t *hoff, int comp, uint8_t *slices,
                                const int64_t *sl_off, const int32_t *expo_q, int32_t *expo_b, const int32_t *tn_b, int S,
                                int F, cudaStream_t st) {
    if (b1 <= b0) return cudaSuccess;
    const int first = comp == 0 ? 1 : 0;  // P' (its exponent and its slices) once, with the first pass
#define NAO_SLICE_NPHI(SS, FF)                                                                                   \
    slice_nphi_kernel<SS, FF, double><<<dim3(b1 - b0, 4 * max_qt + 1), 256, 0, st>>>(                            \
        s, b0, scratch, hoff, comp, slices, sl_off, expo_q, expo_b, tn_b, 10, 1, first)
    NAO_SPLIT_DISPATCH(S, F, NAO_SLICE_NPHI)
#undef NAO_SLICE_NPHI
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !first || max_rt <= 0) return e;
#define NAO_SLICE_NP(SS, FF) \
    slice_np_kernel<SS, FF><<<dim3(b1 - b0, 4 * max_rt), 256, 0, st>>>(s, b0, slices, sl_off, expo_b, tn_b, 1)
    NAO_SPLIT_DISPATCH(S, F, NAO_SLICE_NP)
#undef NAO_SLICE_NP
    return cudaGetLastError();
}

cudaError_t launch_hess_point_expo(const DevSystem &s, int32_t b0, int32_t b1, const double *scratch, const int64_t *hoff,
                                   int32_t *expo4, int64_t n_points, cudaStream_t st) {
    if (b1 <= b0) return cudaSuccess;
    hess_point_expo_kernel<<<b1 - b0, 256, 0, st>>>(s, b0, scratch, hoff, expo4, n_points);
    return cudaGetLastError();
}

// One launch of n_tc_kernel<TN, MODE, F> for the width and digit format at hand.
static cudaError_t launch_n_tc_mode(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work,
                                    const uint8_t *slices, const int64_t *sl_off, const int32_t *expo_q,
                                    const int32_t *expo_b, const void *ev, const int64_t *eoff, int S, int F, int tn,
                                    int mode, int hc, double *hess, int32_t *err, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    if (F == NAO_DIGITS_E4M3 ? tn != 32 : (tn != 32 && !(tn == 48 && S <= 10))) return cudaErrorInvalidValue;
    const size_t sm = split_smem_bytes(S, F);
    const int grid = n_work < sm_count() ? n_work : sm_count();  // persistent: one CTA per SM
#define NAO_N_TC(TNV, M, FF)                                                                                  \
    n_tc_kernel<TNV, M, FF><<<grid, 192, sm, st>>>(s, work, w0, n_work, slices, sl_off, expo_q, expo_b, ev, eoff, S, hc, \
                                                   hess, err)
#define NAO_N_TC_MODES(TNV, FF)             \
    switch (mode) {                         \
        case 0: NAO_N_TC(TNV, 0, FF); break; \
        case 1: NAO_N_TC(TNV, 1, FF); break; \
        case 2: NAO_N_TC(TNV, 2, FF); break; \
        default: NAO_N_TC(TNV, 3, FF); break; \
    }
    if (F == NAO_DIGITS_E4M3) NAO_N_TC_MODES(32, 1)
    else if (tn == 48) NAO_N_TC_MODES(48, 0)
    else NAO_N_TC_MODES(32, 0)
#undef NAO_N_TC_MODES
#undef NAO_N_TC
    return cudaGetLastError();
}

cudaError_t launch_n_tc(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                        const int64_t *sl_off, const int32_t *expo_q, const int32_t *expo_b, const double *scratch, int S,
                        int F, int tn, bool grad, int32_t *err, cudaStream_t st) {
    return launch_n_tc_mode(s, work, w0, n_work, slices, sl_off, expo_q, expo_b, scratch, s.scr_off, S, F, tn, grad ? 1 : 0,
                            0, nullptr, err, st);
}

cudaError_t launch_n_tc_hess(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                             const int64_t *sl_off, const int32_t *expo_q, const int32_t *expo_b, const double *scratch,
                             const int64_t *hoff, int comp, double *hess, int S, int F, int tn, int32_t *err,
                             cudaStream_t st) {
    return launch_n_tc_mode(s, work, w0, n_work, slices, sl_off, expo_q, expo_b, scratch, hoff, S, F, tn,
                            comp == 0 ? 2 : 3, comp, hess, err, st);
}

cudaError_t launch_wn_partial(const DevSystem &s, const DWork *work, int32_t w0, int32_t n_work, double *ne_part,
                              cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    wn_partial_kernel<<<n_work, 256, 0, st>>>(s, work, w0, ne_part);
    return cudaGetLastError();
}

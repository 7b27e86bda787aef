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
#include <cmath>
#include <type_traits>

#include "nao_internal.h"
#include "split_bits.h"
#include "tc_ptx.h"

namespace {

constexpr long long kWaitCycles = 400000000LL;  // ~0.2 s at 2 GHz: bounded mbarrier waits


// Digit extraction works on FP64 bit patterns with integer instructions: on this GPU the FP64
// pipe is ~1/60 of the FP32 rate, and a double-to-int64 conversion per element would make the
// slicing kernels FP64-bound.
using split_bits::abs_bits;

// S balanced base-64 digits (most significant first in dig[0]) of X = round(x 2^(6S-e)),
// |x 2^-e| < 1/2, as exact small-integer floats. From x's bits x = +-m 2^(E-1075) (53-bit m):
// |X| = m 2^-sh with sh = 1075 + e - 6S - E, rounded half up when sh > 0, held as a 128-bit
// integer (hi:lo; more than 64 bits only for S > 10). |X| is cut into 18-bit chunks (three
// digits each), exact in FP32, and the digits are peeled off from the bottom in FP32:
// q = rint(v / 64), d = v - 64 q in [-32, 32], v <- q, the carry q (0 or 1 after a chunk's
// three digits) joining the next chunk. The top digit keeps whatever remains, which the bound
// on |X| keeps in [-32, 32]. Subnormal x and e = -10000 give zeros.
// |X| = round(|x| 2^(6S-e)) as a 128-bit integer (hi:lo) from the bits of x, and the sign of x.
template <int S>
__device__ __forceinline__ void digit_integer(double x, int e, unsigned long long &lo, unsigned long long &hi,
                                              float &sgn) {
    const long long bits = __double_as_longlong(x);
    const int eb = (int)((bits >> 52) & 0x7FF);
    lo = 0;
    hi = 0;
    if (eb != 0 && e > -10000) {
        const unsigned long long m = ((unsigned long long)bits & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
        const int sh = 1075 + e - 6 * S - eb;
        if (sh > 0) {
            lo = sh >= 63 ? 0ULL : (m + (1ULL << (sh - 1))) >> sh;
        } else {
            const int k = -sh;  // <= 6 for S <= 10, <= 18 for S = 12
            lo = m << k;
            hi = k > 0 ? m >> (64 - k) : 0ULL;
        }
    }
    sgn = bits < 0 ? -1.0f : 1.0f;
}

// Chunk c (c = 0, 1, 2: 18 bits; c = 3: the 23 bits from bit 54) of |X| = (hi:lo).
__device__ __forceinline__ uint32_t digit_chunk(unsigned long long lo, unsigned long long hi, int c) {
    return c == 0 ? (uint32_t)(lo & 0x3FFFFULL)
         : c == 1 ? (uint32_t)((lo >> 18) & 0x3FFFFULL)
         : c == 2 ? (uint32_t)((lo >> 36) & 0x3FFFFULL)
                  : (uint32_t)(((lo >> 54) | (hi << 10)) & 0x7FFFFFULL);
}

// The S digits of two values x0, x1 at once (.x and .y of dig[s]) with packed FP32x2 arithmetic.
// The sign is carried in the running value: v starts as sgn |X| mod 2^18 (sgn (2^23 + u) - sgn 2^23,
// one packed FMA, exact), every later chunk enters as + sgn u 2^(18c) at its digit position, and
// the peeling q = rint(v / 64), d = v - 64 q works on signed v as well: rint is odd-symmetric, so
// the digits are those of |X| times the sign.
template <int S>
__device__ __forceinline__ void digits2(double x0, double x1, int e, float2 (&dig)[S]) {
    unsigned long long lo0, hi0, lo1, hi1;
    float s0, s1;
    digit_integer<S>(x0, e, lo0, hi0, s0);
    digit_integer<S>(x1, e, lo1, hi1, s1);
    const float2 sgn = make_float2(s0, s1), nb = make_float2(-8388608.0f * s0, -8388608.0f * s1);
    const float2 inv64 = make_float2(0.015625f, 0.015625f), big = make_float2(12582912.0f, 12582912.0f);
    const float2 nbig = make_float2(-12582912.0f, -12582912.0f), m64 = make_float2(-64.0f, -64.0f);
    auto chunk = [&](int c) {  // sgn u, u < 2^23, exactly
        const float2 u = make_float2(__int_as_float(0x4B000000 | (int)digit_chunk(lo0, hi0, c)),
                                     __int_as_float(0x4B000000 | (int)digit_chunk(lo1, hi1, c)));
        return __ffma2_rn(sgn, u, nb);
    };
    float2 v = chunk(0);
#pragma unroll
    for (int s = S - 1; s >= 0; s--) {
        const int t = S - 1 - s;  // digits already taken
        if (t > 0 && t % 3 == 0) v = __fadd2_rn(v, chunk(t / 3));
        if (s == 0) {
            dig[0] = v;
        } else {
            const float2 q = __fadd2_rn(__ffma2_rn(v, inv64, big), nbig);  // rint(v / 64)
            dig[s] = __ffma2_rn(q, m64, v);
            v = q;
        }
    }
}

// bf16 bit patterns of two small integers held exactly in floats (their low halves are zero).
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    return __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x7632);
}

// 2^E as an FP64 (0 below the normal range).
__device__ __forceinline__ double pow2(int E) {
    if (E < -1022) return 0.0;
    if (E > 1023) E = 1023;
    return __longlong_as_double((long long)(1023 + E) << 52);
}


// ----------------------------------------------------------------------------------------
// Hamiltonian slicing: one CTA per (batch, 64-row tile of basis functions). Columns are
// reordered: the negative-weight ones (v < 0 on the potential part) first, padded to a
// multiple of 16, then the rest, so that B = A and the sign is applied per 16-column K step.
// One warp per row: the row's exponent (a pass over the row), then its digits (a second pass,
// served from L2: the slices are written with evict-first stores so that they do not push the
// rows out).
// ----------------------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(256, S <= 10 ? 5 : 4) slice_h_kernel(DevSystem s, int32_t b0, const double *__restrict__ scratch,
                                                        uint32_t terms, uint8_t *__restrict__ slices,
                                                        const int64_t *__restrict__ sl_off, int32_t *__restrict__ expo,
                                                        int32_t *__restrict__ neg16) {
    __shared__ double sd[4 * NAO_SPLIT_MAX_PPAD];
    __shared__ int sd_eb[4 * NAO_SPLIT_MAX_PPAD];    // biased exponent of sd (0: zero weight)
    __shared__ float sd_m[4 * NAO_SPLIT_MAX_PPAD];   // significand of sd in [1, 2), truncated
    __shared__ short src[4 * NAO_SPLIT_MAX_PPAD + 64];
    __shared__ unsigned char negf[4 * NAO_SPLIT_MAX_PPAD];
    __shared__ int wsum[8];
    const int b = b0 + blockIdx.x, rt = blockIdx.y, m = s.sys.bmol[b];
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const SplitGeom G(P, N, S);
    if (N == 0 || rt >= G.h_slice_tiles()) return;
    const int K = 4 * Ppad, Kp = 64 * G.n_kc;
    const double *E = scratch + s.scr_off[b];
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        const int c = k / Ppad, q = k - c * Ppad;
        const double d = q < P ? split_bits::h_column_weight(s, m, p0 + q, c, terms) : 0.0;
        sd[k] = split_bits::h_column_scale(d);
        const long long sb = __double_as_longlong(sd[k]);
        sd_eb[k] = split_bits::biased_exponent(sb);
        sd_m[k] = split_bits::significand_f(sb);
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
    const int negpad = (total + 15) & ~15;
    for (int k = kb; k < ke; k++) {
        const int pos = negf[k] ? before : negpad + k - before;
        before += negf[k];
        src[pos] = (short)k;
    }
    if (rt == 0 && threadIdx.x == 0) neg16[b] = negpad / 16;
    __syncthreads();
    uint8_t *base = slices + sl_off[b];
    for (int lr = warp; lr < 64; lr += 8) {
        const int r = rt * 64 + lr;
        if (r >= G.R16) break;
        const double *row = E + (int64_t)(r < N ? r : 0) * K;
        int mk = 0;
        if (r < N)
            for (int k = lane; k < K; k += 32) mk = max(mk, split_bits::h_row_key(row[k], sd_eb[k], sd_m[k]));
        mk = __reduce_max_sync(0xffffffffu, mk);
        const int e = r < N ? split_bits::h_row_exponent(mk) : -10000;
        if (lane == 0 && r < N) expo[s.rel_off[b] + r] = e;
        // two consecutive K columns per lane: a warp writes one 128-byte row segment per slice
        for (int kc = 0; kc < G.n_kc; kc++) {
            const int k0 = 64 * kc + 2 * lane;
            const int k0a = src[k0], k0b = src[k0 + 1];
            const double xa = (k0a >= 0 && e > -10000) ? __ldcs(row + k0a) * sd[k0a] : 0.0;
            const double xb = (k0b >= 0 && e > -10000) ? __ldcs(row + k0b) * sd[k0b] : 0.0;
            float2 dg[S];
            digits2<S>(xa, xb, e, dg);
            const uint32_t off = tc::sw128_offset((uint32_t)r, (uint32_t)(2 * lane));
#pragma unroll
            for (int sl = 0; sl < S; sl++)
                __stcs(reinterpret_cast<unsigned int *>(base + G.h_block(sl, kc) + off), pack_bf16x2(dg[sl].x, dg[sl].y));
        }
    }
}

// ----------------------------------------------------------------------------------------
// Density slicing.
// Phi^T: one CTA (8 warps) per (batch, 32-point tile), the point exponents from the
// evaluation. Per 64-function K chunk the CTA stages phi[i][q] (64 x 32, read along the points)
// in shared memory and each warp writes its points' rows along K (two functions per lane, one
// 128-byte row segment per slice). CTAs with blockIdx.y = 0 instead reduce the batch's
// exponent of P' (the upper-triangle tile pairs, read along rows of P).
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ int tile_of(int i, int TN) { return i / TN; }

template <int S>
__global__ void __launch_bounds__(256) slice_nphi_kernel(DevSystem s, int32_t b0, const double *__restrict__ scratch,
                                                        uint8_t *__restrict__ slices, const int64_t *__restrict__ sl_off,
                                                        const int32_t *__restrict__ expo_q, int32_t *__restrict__ expo_b,
                                                        const int32_t *__restrict__ tn_b, int ld_mult, int full) {
    __shared__ double t[32][65];
    __shared__ int red[8];
    const int b = b0 + blockIdx.x;
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    if (N == 0) return;
    const SplitGeom G(P, N, S);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.y == 0) {
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
    const double *E = scratch + s.scr_off[b];  // phi[i][q], row stride ld_mult Ppad (4: rows also hold grad phi)
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
        for (int h = 0; h < 8; h++) {
            const int i = kc * 64 + warp + 8 * h;
            t[lane][warp + 8 * h] = (i < N && qin) ? E[(int64_t)i * ld + q0 + lane] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const int ql = warp * 4 + h, q = q0 + ql;
            if (q >= G.P16) break;
            float2 dg[S];
            digits2<S>(t[ql][2 * lane], t[ql][2 * lane + 1], eq[h], dg);
            const uint32_t off = tc::sw128_offset((uint32_t)q, (uint32_t)(2 * lane));
#pragma unroll
            for (int sl = 0; sl < S; sl++)
                *reinterpret_cast<uint32_t *>(base + G.nA_block(sl, kc) + off) = pack_bf16x2(dg[sl].x, dg[sl].y);
        }
        __syncthreads();
    }
}

// P'_ij = c_IJ P[rel_i][rel_j] over TN-function tiles I = i/TN <= J = j/TN (c_II = 1,
// c_IJ = 2; every (i, j) with c = 1 when full), read from P's upper triangle, with the batch's
// exponent from slice_nphi_kernel. One CTA per (batch, 16 rows j), one warp per row, two
// functions i per lane (one 128-byte row segment per slice).
template <int S>
__global__ void __launch_bounds__(256) slice_np_kernel(DevSystem s, int32_t b0, uint8_t *__restrict__ slices,
                                                      const int64_t *__restrict__ sl_off,
                                                      const int32_t *__restrict__ expo_b,
                                                      const int32_t *__restrict__ tn_b, int full) {
    const int b = b0 + blockIdx.x, m = s.sys.bmol[b];
    const int P = s.batch_off[b + 1] - s.batch_off[b];
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    if (N == 0) return;
    const SplitGeom G(P, N, S);
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
            double xp[2];
#pragma unroll
            for (int hh = 0; hh < 2; hh++) {
                const int i = 64 * kc + 2 * lane + hh;
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
            float2 dg[S];
            digits2<S>(xp[0], xp[1], e, dg);
            const uint32_t off = tc::sw128_offset((uint32_t)j, (uint32_t)(2 * lane));
#pragma unroll
            for (int sl = 0; sl < S; sl++)
                *reinterpret_cast<uint32_t *>(base + G.nB_block(S, sl, kc) + off) = pack_bf16x2(dg[sl].x, dg[sl].y);
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
// at most kMaxRing: 8 for S = 11, 12 (TN = 32), 6 for S = 10 (TN = 48). A deeper ring lets the
// producer's copies run further ahead of the MMAs that wait for them.
__host__ __device__ constexpr int ring_slots(int S) {
    return (int)((kSmemOptin - kStaticSmem - 1024 - 2 * (size_t)S * nao_split_tn(S) * 128) / 16384) < kMaxRing
               ? (int)((kSmemOptin - kStaticSmem - 1024 - 2 * (size_t)S * nao_split_tn(S) * 128) / 16384)
               : kMaxRing;
}

__host__ __device__ constexpr size_t pipe_smem_bytes(int S) {
    return (size_t)ring_slots(S) * 16384 + 2 * (size_t)S * nao_split_tn(S) * 128 + 1024;
}
static_assert(ring_slots(12) >= 4 && ring_slots(10) >= 4 && ring_slots(4) >= 4, "A ring too shallow");
static_assert(pipe_smem_bytes(12) + kStaticSmem <= kSmemOptin && pipe_smem_bytes(10) + kStaticSmem <= kSmemOptin,
              "split pipeline exceeds shared memory");

// Integer recombination of the S group accumulators for 16 columns of this thread's row:
// value = hi 64^-8 + lo 64^-11 + lo2 64^-14 (in units of 2^(e_i + e_j)) with
// hi = sum_{g<=6} M_g 64^(6-g), lo = sum_{7<=g<=9} M_g 64^(9-g), lo2 = sum_{g>=10} M_g 64^(12-g);
// all exact in 64 bits (|M_g| < 2^24).
struct Parts16 {
    long long hi[16], lo[16], lo2[16];
};

template <int TN>
__device__ __forceinline__ void combine16(uint32_t tm_row, int c0, int S, Parts16 &v) {
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
            const int part = g <= 6 ? 0 : (TN == 48 || g <= 9 ? 1 : 2);  // TN = 48: S <= 10, no lo2
            const long long w = 1LL << (6 * (part == 0 ? 6 - g : (part == 1 ? 9 - g : 12 - g)));
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

template <int TN>
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
    const SplitGeom G(P, h.N, S);
    const uint8_t *base = slices + sl_off[h.b];
    h.blk = (size_t)G.R16 * 128;
    h.a0 = base + (size_t)it.ti * 128 * 128;
    h.b0 = base + (size_t)it.tj * TN * 128;
    h.a_bytes = (uint32_t)min(128, G.R16 - it.ti * 128) * 128u;
    h.b_bytes = (uint32_t)min(TN, G.R16 - it.tj * TN) * 128u;
    h.n_kc = G.n_kc;
    nao_split_h_seg_range(G.n_kc, nao_split_h_nseg(P, S), it.pad, S, h.kc0, h.kc1);
    h.neg16 = neg16[h.b];
    return h;
}

template <int TN>
__global__ void __launch_bounds__(192, 1)
    h_tc_kernel(DevSystem s, const HWork *__restrict__ work, int32_t w0, int32_t n_work, const uint8_t *__restrict__ slices,
                const int64_t *__restrict__ sl_off, const int32_t *__restrict__ expo,
                const int32_t *__restrict__ neg16, int S, int scatter, int32_t *__restrict__ err) {
    constexpr uint32_t B_BLOCK = TN * 128;
    extern __shared__ uint8_t smem_dyn[];
    __shared__ PPipe pp;
    uint8_t *smem = align1024(smem_dyn);
    const int RING = ring_slots(S);
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
                const HItem h = h_item<TN>(s, work, w0 + w, slices, sl_off, neg16, S);
                const bool more = w + (int)gridDim.x < n_work;
                HItem hn = h;
                if (more) hn = h_item<TN>(s, work, w0 + w + gridDim.x, slices, sl_off, neg16, S);
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
                const HItem h = h_item<TN>(s, work, w0 + w, slices, sl_off, neg16, S);
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
                        // pairs (sa, t = 0 .. S-1-sa): one MMA per 16-column K step (two above N = 256)
                        const int ncols = TN * (S - sa);
                        for (int n0 = 0; n0 < ncols; n0 += 256) {
                            const int nn = ncols - n0 < 256 ? ncols - n0 : 256;
                            const uint32_t idesc = tc::idesc_bf16_f32(128, nn);
                            const uint64_t bd = tc::sdesc_sw128(tc::smem_addr(bset + (size_t)n0 * 128));
                            const uint32_t dt = tm + (uint32_t)(sa * TN + n0);
#pragma unroll
                            for (int ks = 0; ks < 4; ks++) {
                                const uint32_t id = (kc * 4 + ks < h.neg16) ? (idesc | (1u << 14)) : idesc;
                                tc::mma_bf16(dt, ad + 2 * ks, bd + 2 * ks, id, (first | sa | ks) ? 1u : 0u);
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
            const HItem h = h_item<TN>(s, work, w0 + w, slices, sl_off, neg16, S);
            if (*abort || !tc::mbar_wait(&pp.acc_full, t & 1, kWaitCycles)) { *abort = 1; break; }
            tc::fence_after_sync();
            const int i = h.ti * 128 + warp * 32 + lane;
            const bool row_ok = i < h.N;
            const int32_t *rel = s.rel_idx + s.rel_off[h.b];
            const int32_t *ex = expo + s.rel_off[h.b];
            const int ei = row_ok ? ex[i] : -10000;
            // h_ij as one 64-bit integer, exact as hi 2^18 + lo' where |hi| < 2^44, else
            // 4 hi + round(lo' / 2^16) (|4 hi| >= 2^46: relative error <= 2^-47), with lo' = lo +
            // round(lo2 / 2^18): the groups g >= 10 that only S = 11, 12 have are folded into lo at
            // a cost of at most half a unit of lo, 2^-67 of 2^(e_i + e_j), far below the split's own
            // truncation. The integers are formed before tensor memory is handed back, the
            // conversion and the product by 2^(e_i + e_j - 66 or - 50) after.
            long long val[TN];
            uint64_t small_mask = 0;
#pragma unroll
            for (int c0 = 0; c0 < TN; c0 += 16) {
                Parts16 v;
                combine16<TN>(tm_row, c0, S, v);
#pragma unroll
                for (int jj = 0; jj < 16; jj++) {
                    const long long hi = v.hi[jj], lo = v.lo[jj] + ((v.lo2[jj] + (1LL << 17)) >> 18);
                    const bool small = hi > -(1LL << 44) && hi < (1LL << 44);
                    val[c0 + jj] = small ? (hi << 18) + lo : (hi << 2) + ((lo + (1LL << 15)) >> 16);
                    small_mask |= (uint64_t)small << (c0 + jj);
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
                        const double x = (ei > -10000 && ej > -10000)
                                             ? (double)val[jj] * pow2(ei + ej - (((small_mask >> jj) & 1) ? 66 : 50))
                                             : 0.0;
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

template <int TN>
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
    const SplitGeom G(h.P, h.N, S, TN);
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
template <int TN, bool GRADN>
__device__ __forceinline__ int n_item_kc(const NItem &h, int J) {
    const int nk = GRADN ? h.n_kcN : ((J + 1) * TN + 63) / 64;
    return nk < h.n_kcN ? nk : h.n_kcN;
}

template <int TN, bool GRADN>
__global__ void __launch_bounds__(192, 1)
    n_tc_kernel(DevSystem s, const HWork *__restrict__ work, int32_t w0, int32_t n_work, const uint8_t *__restrict__ slices,
                const int64_t *__restrict__ sl_off, const int32_t *__restrict__ expo_q,
                const int32_t *__restrict__ expo_b, const double *__restrict__ scratch, int S,
                int32_t *__restrict__ err) {
    constexpr uint32_t B_BLOCK = TN * 128;
    extern __shared__ uint8_t smem_dyn[];
    __shared__ PPipe pp;
    uint8_t *smem = align1024(smem_dyn);
    const int RING = ring_slots(S);
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
                const NItem h = n_item<TN>(s, work, w0 + w, slices, sl_off, S);
                for (int J = 0; J < h.nJ && !*abort; J++) {
                    const int nk = n_item_kc<TN, GRADN>(h, J);
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
                const NItem h = n_item<TN>(s, work, w0 + w, slices, sl_off, S);
                for (int J = 0; J < h.nJ && !*abort; J++, t++) {
                    const int nk = n_item_kc<TN, GRADN>(h, J);
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
                            // pairs (sa, t = 0 .. S-1-sa): one MMA per 16-column K step (two above N = 256)
                            const int ncols = TN * (S - sa);
                            for (int n0 = 0; n0 < ncols; n0 += 256) {
                                const int nn = ncols - n0 < 256 ? ncols - n0 : 256;
                                const uint32_t idesc = tc::idesc_bf16_f32(128, nn);
                                const uint64_t bd = tc::sdesc_sw128(tc::smem_addr(bset + (size_t)n0 * 128));
                                const uint32_t dt = tm + (uint32_t)(sa * TN + n0);
#pragma unroll
                                for (int ks = 0; ks < 4; ks++)
                                    tc::mma_bf16(dt, ad + 2 * ks, bd + 2 * ks, idesc, (kc | sa | ks) ? 1u : 0u);
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
            const NItem h = n_item<TN>(s, work, w0 + w, slices, sl_off, S);
            const int q = h.ti * 128 + warp * 32 + lane;
            const bool row_ok = q < h.P;
            const double *E = scratch + s.scr_off[h.b];
            const int64_t ld = GRADN ? 4 * (int64_t)h.Ppad : (int64_t)h.Ppad;
            // sum_j T_qj phi_qj (and grad phi) in units of 2^(e_q + e_b - 50): each T_qj as one
            // 64-bit integer in those units, 4 hi + round(lo' / 2^16) (|4 hi| < 2^62.03; lo' = lo +
            // round(lo2 / 2^18) folds the groups g >= 10 of S = 11, 12), rounded by at most 2^-1
            // unit: the order of the split's truncation at S = 10 (the dropped groups g >= S reach
            // K (S + 1) 2^(e_q + e_b - 6S - 2)) and below the FP64 evaluation's rounding in n. Then
            // one conversion and one FMA per product, all integer work done before tensor memory is
            // handed back (no FP64 arithmetic on that path).
            double part = 0.0, gpart[3] = {0.0, 0.0, 0.0};
            for (int J = 0; J < h.nJ; J++, t++) {
                if (*abort || !tc::mbar_wait(&pp.acc_full, t & 1, kWaitCycles)) { *abort = 1; break; }
                tc::fence_after_sync();
                long long val[TN];
#pragma unroll
                for (int c0 = 0; c0 < TN; c0 += 16) {
                    Parts16 v;
                    combine16<TN>(tm_row, c0, S, v);
#pragma unroll
                    for (int jj = 0; jj < 16; jj++) {
                        const long long lo = v.lo[jj] + ((v.lo2[jj] + (1LL << 17)) >> 18);  // lo2: S = 11, 12
                        val[c0 + jj] = (v.hi[jj] << 2) + ((lo + (1LL << 15)) >> 16);
                    }
                }
                // tensor memory is free for the next tile
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&pp.acc_empty);
                if (row_ok) {
                    // the next tile's rows of phi towards L2 while this tile's products run
                    if (J + 1 < h.nJ) {
                        const double *fn = E + (int64_t)(J + 1) * TN * ld + q;
                        const int jn1 = min(TN, h.N - (J + 1) * TN);
                        for (int jj = 0; jj < jn1; jj++) asm volatile("prefetch.global.L2 [%0];" ::"l"(fn + jj * ld));
                    }
                    const int jn = min(TN, h.N - J * TN);
                    const double *f = E + (int64_t)J * TN * ld + q;
#pragma unroll
                    for (int jj = 0; jj < TN; jj++) {
                        if (jj < jn) {
                            const double vj = (double)val[jj];
                            part = fma(vj, f[jj * ld], part);
                            if (GRADN)
#pragma unroll
                                for (int d = 0; d < 3; d++) gpart[d] = fma(vj, f[jj * ld + (d + 1) * h.Ppad], gpart[d]);
                        }
                    }
                }
            }
            if (*abort) break;
            if (row_ok) {
                const int eq = expo_q[h.p0 + q], eb = expo_b[h.b];
                const bool live = eq > -10000 && eb > -10000;
                const double sc = pow2(eq + eb - 50);
                *n_at(s, h.m, h.p0 + q) = live ? part * sc : 0.0;
                if (GRADN)
#pragma unroll
                    for (int d = 0; d < 3; d++) *gn_at(s, h.m, h.p0 + q, d) = live ? 2.0 * gpart[d] * sc : 0.0;
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

}  // namespace

size_t split_smem_bytes(int S) { return pipe_smem_bytes(S); }

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
    for (int S = 4; S <= NAO_SPLIT_MAX_SLICES; S++) bytes = split_smem_bytes(S) > bytes ? split_smem_bytes(S) : bytes;
    const void *fns[6] = {(const void *)h_tc_kernel<48>, (const void *)h_tc_kernel<32>,
                          (const void *)n_tc_kernel<48, false>, (const void *)n_tc_kernel<32, false>,
                          (const void *)n_tc_kernel<48, true>, (const void *)n_tc_kernel<32, true>};
    for (const void *f : fns) {
        const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

#define NAO_SPLIT_DISPATCH(S, CALL)                  \
    switch (S) {                                    \
        case 4: CALL(4); break;                     \
        case 5: CALL(5); break;                     \
        case 6: CALL(6); break;                     \
        case 7: CALL(7); break;                     \
        case 8: CALL(8); break;                     \
        case 9: CALL(9); break;                     \
        case 10: CALL(10); break;                   \
        case 11: CALL(11); break;                   \
        default: CALL(12); break;                   \
    }

cudaError_t launch_slice_h(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_rt, const double *scratch,
                           uint32_t terms, uint8_t *slices, const int64_t *sl_off, int32_t *expo, int32_t *neg16, int S,
                           cudaStream_t st) {
    if (b1 <= b0 || max_rt <= 0) return cudaSuccess;
#define NAO_SLICE_H(SS) \
    slice_h_kernel<SS><<<dim3(b1 - b0, max_rt), 256, 0, st>>>(s, b0, scratch, terms, slices, sl_off, expo, neg16)
    NAO_SPLIT_DISPATCH(S, NAO_SLICE_H)
#undef NAO_SLICE_H
    return cudaGetLastError();
}

cudaError_t launch_h_tc(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                        const int64_t *sl_off, const int32_t *expo, const int32_t *neg16, int S, int tn, int scatter,
                        int32_t *err, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    const int grid = n_work < sm_count() ? n_work : sm_count();  // persistent: one CTA per SM
    if (tn == 48 && S <= 10)
        h_tc_kernel<48><<<grid, 192, split_smem_bytes(S), st>>>(s, work, w0, n_work, slices, sl_off, expo, neg16, S,
                                                               scatter, err);
    else if (tn == 32)
        h_tc_kernel<32><<<grid, 192, split_smem_bytes(S), st>>>(s, work, w0, n_work, slices, sl_off, expo, neg16, S,
                                                               scatter, err);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_slice_n(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_qt, int32_t max_rt,
                           const double *scratch, uint8_t *slices, const int64_t *sl_off, const int32_t *expo_q,
                           int32_t *expo_b, const int32_t *tn_b, int S, bool grad, cudaStream_t st) {
    if (b1 <= b0) return cudaSuccess;
    // y = 0: the exponent of P'; y >= 1: 32-point tiles (128 max_qt >= P16)
#define NAO_SLICE_NPHI(SS)                                                                                   \
    slice_nphi_kernel<SS><<<dim3(b1 - b0, 4 * max_qt + 1), 256, 0, st>>>(s, b0, scratch, slices, sl_off, expo_q, \
                                                                         expo_b, tn_b, grad ? 4 : 1, grad ? 1 : 0)
    NAO_SPLIT_DISPATCH(S, NAO_SLICE_NPHI)
#undef NAO_SLICE_NPHI
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || max_rt <= 0) return e;
    // 16 rows per CTA (64 max_rt >= R16)
#define NAO_SLICE_NP(SS) \
    slice_np_kernel<SS><<<dim3(b1 - b0, 4 * max_rt), 256, 0, st>>>(s, b0, slices, sl_off, expo_b, tn_b, grad ? 1 : 0)
    NAO_SPLIT_DISPATCH(S, NAO_SLICE_NP)
#undef NAO_SLICE_NP
    return cudaGetLastError();
}

cudaError_t launch_n_tc(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                        const int64_t *sl_off, const int32_t *expo_q, const int32_t *expo_b, const double *scratch, int S,
                        int tn, bool grad, int32_t *err, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    if (tn != 32 && !(tn == 48 && S <= 10)) return cudaErrorInvalidValue;
    const size_t sm = split_smem_bytes(S);
    const int grid = n_work < sm_count() ? n_work : sm_count();  // persistent: one CTA per SM
#define NAO_N_TC(TNV, G) \
    n_tc_kernel<TNV, G><<<grid, 192, sm, st>>>(s, work, w0, n_work, slices, sl_off, expo_q, expo_b, scratch, S, err)
    if (tn == 48 && grad) NAO_N_TC(48, true);
    else if (tn == 48) NAO_N_TC(48, false);
    else if (grad) NAO_N_TC(32, true);
    else NAO_N_TC(32, false);
#undef NAO_N_TC
    return cudaGetLastError();
}

cudaError_t launch_wn_partial(const DevSystem &s, const DWork *work, int32_t w0, int32_t n_work, double *ne_part,
                              cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    wn_partial_kernel<<<n_work, 256, 0, st>>>(s, work, w0, ne_part);
    return cudaGetLastError();
}

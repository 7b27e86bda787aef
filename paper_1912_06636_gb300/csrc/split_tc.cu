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

#include "nao_internal.h"
#include "tc_ptx.h"

namespace {

constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: bounded mbarrier waits

// bf16 bit pattern of a small integer (|d| <= 256 is exact).
__device__ __forceinline__ uint32_t bf16_bits(int d) { return __float_as_uint((float)d) >> 16; }

// S balanced base-64 digits of X = round(Y), |Y| < 2^(6S-1) (most significant first in
// dig[0]), in integer arithmetic. The S-1 lower digits are taken in [-32, 31]; the top digit
// is what remains, which the bound on |X| keeps in [-32, 32] (it must not be reduced modulo
// 64, or a carry would be lost). For S > 10, X may need more than 64 bits; but an FP64 Y with
// |Y| >= 2^63 is an integer m 2^k (53-bit m, k >= 11), so X = (m 2^(k mod 6)) 64^(k/6): the
// last k/6 digits are zero and the others are those of m 2^(k mod 6) < 2^59.
template <int S>
__device__ __forceinline__ void digits(double Y, int (&dig)[S]) {
    long long X;
    int q = 0;  // trailing zero digits
    if (S <= 10 || fabs(Y) < 9223372036854775808.0) {
        X = __double2ll_rn(Y);
    } else {
        const long long bits = __double_as_longlong(Y);
        const int k = (int)((bits >> 52) & 0x7FF) - 1075;  // Y = +-m 2^k
        const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
        q = k / 6;
        X = m << (k - 6 * q);
        if (bits < 0) X = -X;
    }
#pragma unroll
    for (int s = S - 1; s >= 1; s--) {
        if (s >= S - q) {
            dig[s] = 0;
        } else {
            const int d = (int)(((X + 32) & 63LL)) - 32;
            dig[s] = d;
            X = (X - d) >> 6;
        }
    }
    dig[0] = (int)X;
}

// Exponent e with max * 2^-e in [0.25, 0.5); rows whose magnitude is below 2^-900 are taken
// as zero (flag -10000).
__device__ __forceinline__ int row_exponent(double mx) {
    if (!(mx > 0.0)) return -10000;
    int ex;
    frexp(mx, &ex);
    return ex < -900 ? -10000 : ex + 1;
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
// ----------------------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(256) slice_h_kernel(DevSystem s, int32_t b0, const double *__restrict__ scratch,
                                                     uint32_t terms, uint8_t *__restrict__ slices,
                                                     const int64_t *__restrict__ sl_off, int32_t *__restrict__ expo,
                                                     int32_t *__restrict__ neg16) {
    __shared__ double sd[4 * NAO_SPLIT_MAX_PPAD];
    __shared__ short src[4 * NAO_SPLIT_MAX_PPAD + 64];
    __shared__ unsigned char negf[4 * NAO_SPLIT_MAX_PPAD];
    __shared__ int wsum[8];
    __shared__ int ex_s[64];
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
        const double w = q < P ? s.pw[p0 + q] : 0.0;
        double d;
        if (c == 0) d = (terms & NAO_TERM_POTENTIAL) && q < P ? w * v_at(s, m, p0 + q) : 0.0;
        else d = (terms & NAO_TERM_KINETIC) ? 0.5 * w : 0.0;
        sd[k] = sqrt(fabs(d));
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
    for (int lr = warp; lr < 64; lr += 8) {
        const int r = rt * 64 + lr;
        double mx = 0.0;
        if (r < N)
            for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(E[(int64_t)r * K + k] * sd[k]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            const int e = row_exponent(mx);
            ex_s[lr] = e;
            if (r < N) expo[s.rel_off[b] + r] = e;
        }
    }
    __syncthreads();
    uint8_t *base = slices + sl_off[b];
    const int groups = Kp / 8;
    for (int u = threadIdx.x; u < 64 * groups; u += blockDim.x) {
        const int lr = u / groups, k0 = (u - lr * groups) * 8;
        const int r = rt * 64 + lr;
        if (r >= G.R16) continue;
        const int e = ex_s[lr];
        int dg[8][S];
        const double scale = (r < N && e > -10000) ? pow2(6 * S - e) : 0.0;
        const double *row = E + (int64_t)(r < N ? r : 0) * K;
#pragma unroll
        for (int h = 0; h < 8; h++) {
            const int kk = src[k0 + h];
            const double x = (kk >= 0 && scale != 0.0) ? row[kk] * sd[kk] : 0.0;
            digits<S>(x * scale, dg[h]);
        }
        const int kc = k0 >> 6;
        const uint32_t off = tc::sw128_offset((uint32_t)r, (uint32_t)(k0 & 63));
#pragma unroll
        for (int sl = 0; sl < S; sl++) {
            uint4 va;
            va.x = bf16_bits(dg[0][sl]) | (bf16_bits(dg[1][sl]) << 16);
            va.y = bf16_bits(dg[2][sl]) | (bf16_bits(dg[3][sl]) << 16);
            va.z = bf16_bits(dg[4][sl]) | (bf16_bits(dg[5][sl]) << 16);
            va.w = bf16_bits(dg[6][sl]) | (bf16_bits(dg[7][sl]) << 16);
            *reinterpret_cast<uint4 *>(base + G.h_block(sl, kc) + off) = va;
        }
    }
}

// ----------------------------------------------------------------------------------------
// Density slicing. Phi^T: one CTA (128 threads, one point each) per (batch, 128-point tile).
// ----------------------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(128) slice_nphi_kernel(DevSystem s, int32_t b0, const double *__restrict__ scratch,
                                                        uint8_t *__restrict__ slices, const int64_t *__restrict__ sl_off,
                                                        int32_t *__restrict__ expo_q) {
    const int b = b0 + blockIdx.x, qt = blockIdx.y;
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const SplitGeom G(P, N, S);
    const int q = qt * 128 + threadIdx.x;
    if (N == 0 || q >= G.P16) return;
    const double *E = scratch + s.scr_off[b];  // phi[i][q], stride Ppad
    double mx = 0.0;
    if (q < P)
        for (int i = 0; i < N; i++) mx = fmax(mx, fabs(E[(int64_t)i * Ppad + q]));
    const int e = q < P ? row_exponent(mx) : -10000;
    if (q < P) expo_q[p0 + q] = e;
    const double scale = e > -10000 ? pow2(6 * S - e) : 0.0;
    uint8_t *base = slices + sl_off[b];
    for (int i0 = 0; i0 < G.n_kcN * 64; i0 += 8) {
        int dg[8][S];
#pragma unroll
        for (int h = 0; h < 8; h++) {
            const int i = i0 + h;
            const double x = (scale != 0.0 && i < N) ? E[(int64_t)i * Ppad + q] : 0.0;
            digits<S>(x * scale, dg[h]);
        }
        const int kc = i0 >> 6;
        const uint32_t off = tc::sw128_offset((uint32_t)q, (uint32_t)(i0 & 63));
#pragma unroll
        for (int sl = 0; sl < S; sl++) {
            uint4 va;
            va.x = bf16_bits(dg[0][sl]) | (bf16_bits(dg[1][sl]) << 16);
            va.y = bf16_bits(dg[2][sl]) | (bf16_bits(dg[3][sl]) << 16);
            va.z = bf16_bits(dg[4][sl]) | (bf16_bits(dg[5][sl]) << 16);
            va.w = bf16_bits(dg[6][sl]) | (bf16_bits(dg[7][sl]) << 16);
            *reinterpret_cast<uint4 *>(base + G.nA_block(sl, kc) + off) = va;
        }
    }
}

// P'_ij = c_IJ P[rel_i][rel_j] over TN-function tiles I = i/TN <= J = j/TN (c_II = 1,
// c_IJ = 2), read from P's upper triangle. One CTA per batch: a per-batch exponent, then the
// digits of rows j (TN-row blocks), K = i (chunks of 64).
template <int S>
__global__ void __launch_bounds__(256) slice_np_kernel(DevSystem s, int32_t b0, uint8_t *__restrict__ slices,
                                                      const int64_t *__restrict__ sl_off, int32_t *__restrict__ expo_b) {
    __shared__ double red[8];
    __shared__ int e_sh;
    const int b = b0 + blockIdx.x, m = s.sys.bmol[b];
    const int P = s.batch_off[b + 1] - s.batch_off[b];
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    if (N == 0) return;
    const SplitGeom G(P, N, S);
    const int32_t *rel = s.rel_idx + s.rel_off[b];
    constexpr int TN = nao_split_tn(S);
    auto pval = [&](int i, int j) -> double {
        if (i >= N || j >= N || i / TN > j / TN) return 0.0;
        int64_t gi = rel[i], gj = rel[j];
        if (gi > gj) { const int64_t t = gi; gi = gj; gj = t; }
        const double c = i / TN < j / TN ? 2.0 : 1.0;
        return c * p_elem(s, m, gi, gj);
    };
    double mx = 0.0;
    for (int u = threadIdx.x; u < N * N; u += blockDim.x) mx = fmax(mx, fabs(pval(u / N, u % N)));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < 8; w++) m = fmax(m, red[w]);
        e_sh = row_exponent(m);
        expo_b[b] = e_sh;
    }
    __syncthreads();
    const int e = e_sh;
    const double scale = e > -10000 ? pow2(6 * S - e) : 0.0;
    uint8_t *base = slices + sl_off[b];
    const int groups = G.n_kcN * 8;  // 8-wide groups along K = i
    for (int u = threadIdx.x; u < G.R16 * groups; u += blockDim.x) {
        const int j = u / groups, i0 = (u - j * groups) * 8;
        int dg[8][S];
#pragma unroll
        for (int h = 0; h < 8; h++) digits<S>(pval(i0 + h, j) * scale, dg[h]);
        const int kc = i0 >> 6;
        const uint32_t off = tc::sw128_offset((uint32_t)j, (uint32_t)(i0 & 63));
#pragma unroll
        for (int sl = 0; sl < S; sl++) {
            uint4 vb;
            vb.x = bf16_bits(dg[0][sl]) | (bf16_bits(dg[1][sl]) << 16);
            vb.y = bf16_bits(dg[2][sl]) | (bf16_bits(dg[3][sl]) << 16);
            vb.z = bf16_bits(dg[4][sl]) | (bf16_bits(dg[5][sl]) << 16);
            vb.w = bf16_bits(dg[6][sl]) | (bf16_bits(dg[7][sl]) << 16);
            *reinterpret_cast<uint4 *>(base + G.nB_block(S, sl, kc) + off) = vb;
        }
    }
}

// ----------------------------------------------------------------------------------------
// Slice-product pipeline. Shared memory: a ring of 4 A-tile buffers (128 rows x 64 bf16,
// 16 KB, one slice of one K chunk each) and two sets of S B-tile buffers (TN rows, TN x 128 B).
// Producer (warp 0, one lane): for each K chunk, the S B slices into B set kc % 2, then the
// S A slices one by one into the ring, each copy a single bulk (TMA) transfer completing on a
// "full" mbarrier. MMA issuer (warp 1, one lane): for each A slice s, the pairs (s, t) with
// s + t < S, four 128xTNx16 tcgen05.mma each into accumulator group s + t (tensor-memory
// columns TN (s + t) ...); commits release A buffers and B sets back to the producer through
// "empty" mbarriers. The 16-column K steps with index < neg16 negate B (descriptor bit 14).
// Every wait is bounded; on a timeout the CTA records NAO_ERR_TIMEOUT and skips its epilogue.
// ----------------------------------------------------------------------------------------
constexpr int RING = 4;

struct Pipe {
    uint64_t fullA[RING], emptyA[RING], fullB[2], emptyB[2], done;
    uint32_t tmem;
    int abort;
};

struct LoopArgs {
    const uint8_t *a0;  // A tile (slice s, chunk kc) at a0 + s a_s + kc a_kc, a_bytes long
    size_t a_s, a_kc;
    const uint8_t *b0;  // B tile (slice t, chunk kc) at b0 + t b_s + kc b_kc, b_bytes long
    size_t b_s, b_kc;
    uint32_t a_bytes, b_bytes;  // <= 16 KB and TN x 128 B (the last tile of an operand is short)
    int n_kc, neg16, S;
};

__host__ __device__ constexpr size_t pipe_smem_bytes(int S) {
    return (size_t)RING * 16384 + 2 * (size_t)S * nao_split_tn(S) * 128 + 1024;
}

template <int TN>
__device__ __forceinline__ void pipe_producer(Pipe &p, uint8_t *sA, uint8_t *sB, const LoopArgs &L) {
    constexpr uint32_t B_BLOCK = TN * 128;
    const int S = L.S;
    for (int kc = 0; kc < L.n_kc; kc++) {
        const int bb = kc & 1, ub = kc >> 1;
        if (ub >= 1 && !tc::mbar_wait(&p.emptyB[bb], (ub - 1) & 1, kWaitCycles)) { p.abort = 1; return; }
        tc::mbar_arrive_expect_tx(&p.fullB[bb], (uint32_t)S * L.b_bytes);
        for (int t = 0; t < S; t++)
            tc::bulk_g2s(sB + ((size_t)bb * S + t) * B_BLOCK, L.b0 + t * L.b_s + kc * L.b_kc, L.b_bytes, &p.fullB[bb]);
        for (int sa = 0; sa < S; sa++) {
            const int idx = kc * S + sa, a = idx % RING, ua = idx / RING;
            if (ua >= 1 && !tc::mbar_wait(&p.emptyA[a], (ua - 1) & 1, kWaitCycles)) { p.abort = 1; return; }
            tc::mbar_arrive_expect_tx(&p.fullA[a], L.a_bytes);
            tc::bulk_g2s(sA + (size_t)a * 16384, L.a0 + sa * L.a_s + kc * L.a_kc, L.a_bytes, &p.fullA[a]);
        }
        if (*(volatile int *)&p.abort) return;
    }
}

template <int TN>
__device__ __forceinline__ void pipe_mma(Pipe &p, uint8_t *sA, uint8_t *sB, uint32_t tm, const LoopArgs &L) {
    constexpr uint32_t B_BLOCK = TN * 128;
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, TN);
    const int S = L.S;
    for (int kc = 0; kc < L.n_kc; kc++) {
        const int bb = kc & 1, ub = kc >> 1;
        // on a timeout: flag it, and still commit "done" so the teardown waits for issued MMAs
        if (!tc::mbar_wait(&p.fullB[bb], ub & 1, kWaitCycles)) { p.abort = 1; tc::mma_commit(&p.done); return; }
        for (int sa = 0; sa < S; sa++) {
            const int idx = kc * S + sa, a = idx % RING, ua = idx / RING;
            if (!tc::mbar_wait(&p.fullA[a], ua & 1, kWaitCycles)) { p.abort = 1; tc::mma_commit(&p.done); return; }
            tc::fence_after_sync();
            const uint64_t ad = tc::sdesc_sw128(tc::smem_addr(sA + (size_t)a * 16384));
            for (int tb = 0; sa + tb < S; tb++) {
                const uint64_t bd = tc::sdesc_sw128(tc::smem_addr(sB + ((size_t)bb * S + tb) * B_BLOCK));
                const uint32_t dt = tm + (uint32_t)((sa + tb) * TN);
#pragma unroll
                for (int ks = 0; ks < 4; ks++) {
                    const uint32_t id = (kc * 4 + ks < L.neg16) ? (idesc | (1u << 14)) : idesc;
                    tc::mma_bf16(dt, ad + 2 * ks, bd + 2 * ks, id, (kc | sa | ks) ? 1u : 0u);
                }
            }
            tc::mma_commit(&p.emptyA[a]);
        }
        tc::mma_commit(&p.emptyB[bb]);
    }
    tc::mma_commit(&p.done);
}

// Runs the pipeline; on return (all threads) the accumulators are complete unless p.abort.
template <int TN>
__device__ __forceinline__ void pipe_run(Pipe &p, uint8_t *smem, uint32_t tm, const LoopArgs &L, int32_t *err) {
    uint8_t *sA = smem, *sB = smem + (size_t)RING * 16384;
    if (threadIdx.x == 0) pipe_producer<TN>(p, sA, sB, L);
    else if (threadIdx.x == 32) pipe_mma<TN>(p, sA, sB, tm, L);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!tc::mbar_wait(&p.done, 0, kWaitCycles)) p.abort = 1;
        if (p.abort) atomicExch(err, (int)NAO_ERR_TIMEOUT);
    }
    __syncthreads();
    tc::fence_after_sync();
}

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
    for (int g = 0; g < S; g++) {
        uint32_t r[16];
        tc::tmem_ld16(tm_row + (uint32_t)(g * TN + c0), r);
        tc::tmem_ld_wait();
        const int part = g <= 6 ? 0 : (TN == 48 || g <= 9 ? 1 : 2);  // TN = 48: S <= 10, no lo2
        const long long w = 1LL << (6 * (part == 0 ? 6 - g : (part == 1 ? 9 - g : 12 - g)));
#pragma unroll
        for (int jj = 0; jj < 16; jj++) {
            const long long m = (long long)__float2int_rn(__uint_as_float(r[jj]));
            if (part == 0) v.hi[jj] += m * w;
            else if (part == 1) v.lo[jj] += m * w;
            else v.lo2[jj] += m * w;
        }
    }
}

// 2^(e_i + e_j) (hi 64^-8 + lo 64^-11 + lo2 64^-14)
__device__ __forceinline__ double recombine(long long hi, long long lo, long long lo2, int eij) {
    return fma((double)hi, pow2(eij - 48), fma((double)lo, pow2(eij - 66), (double)lo2 * pow2(eij - 84)));
}

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ uint32_t tc_setup(Pipe &p) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int i = 0; i < RING; i++) {
            tc::mbar_init(&p.fullA[i], 1);
            tc::mbar_init(&p.emptyA[i], 1);
        }
        for (int i = 0; i < 2; i++) {
            tc::mbar_init(&p.fullB[i], 1);
            tc::mbar_init(&p.emptyB[i], 1);
        }
        tc::mbar_init(&p.done, 1);
        tc::fence_mbar_init();
        p.abort = 0;
    }
    __syncwarp();
    if (warp == 0) {
        tc::tmem_alloc(&p.tmem, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    return p.tmem;
}

__device__ __forceinline__ void tc_teardown(uint32_t tm) {
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(tm, 512);
}

template <int TN>
__global__ void __launch_bounds__(128, 1) h_tc_kernel(DevSystem s, const HWork *__restrict__ work, int32_t w0,
                                                     const uint8_t *__restrict__ slices, const int64_t *__restrict__ sl_off,
                                                     const int32_t *__restrict__ expo, const int32_t *__restrict__ neg16,
                                                     int S, int32_t *__restrict__ err) {
    extern __shared__ uint8_t smem_dyn[];
    __shared__ Pipe pp;
    uint8_t *smem = align1024(smem_dyn);
    const HWork it = work[w0 + blockIdx.x];  // batch, 128-row tile, TN-column tile
    const int b = it.batch, m = s.sys.bmol[b];
    const int P = s.batch_off[b + 1] - s.batch_off[b];
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const SplitGeom G(P, N, S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tm = tc_setup(pp);
    const uint8_t *base = slices + sl_off[b];
    const size_t blk = (size_t)G.R16 * 128;
    LoopArgs L;
    L.a0 = base + (size_t)it.ti * 128 * 128;
    L.b0 = base + (size_t)it.tj * TN * 128;
    L.a_s = L.b_s = (size_t)G.n_kc * blk;
    L.a_kc = L.b_kc = blk;
    L.a_bytes = (uint32_t)min(128, G.R16 - it.ti * 128) * 128u;
    L.b_bytes = (uint32_t)min(TN, G.R16 - it.tj * TN) * 128u;
    L.n_kc = G.n_kc;
    L.neg16 = neg16[b];
    L.S = S;
    pipe_run<TN>(pp, smem, tm, L, err);
    if (!pp.abort) {
        const int i = it.ti * 128 + warp * 32 + lane;
        const bool row_ok = i < N;
        const int32_t *rel = s.rel_idx + s.rel_off[b];
        const int32_t *ex = expo + s.rel_off[b];
        const int ei = row_ok ? ex[i] : -10000;
        const int64_t gi = row_ok ? rel[i] : 0;
        const uint32_t tm_row = tm + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < TN; c0 += 16) {
            Parts16 v;
            combine16<TN>(tm_row, c0, S, v);
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const int j = it.tj * TN + c0 + jj;
                if (!row_ok || j >= N || j < i) continue;
                const int ej = ex[j];
                if (ei <= -10000 || ej <= -10000) continue;
                atomicAdd(h_elem(s, m, gi, rel[j]), recombine(v.hi[jj], v.lo[jj], v.lo2[jj], ei + ej));
            }
        }
    }
    tc_teardown(tm);
}

template <int TN>
__global__ void __launch_bounds__(128, 1) n_tc_kernel(DevSystem s, const HWork *__restrict__ work, int32_t w0,
                                                     const uint8_t *__restrict__ slices, const int64_t *__restrict__ sl_off,
                                                     const int32_t *__restrict__ expo_q, const int32_t *__restrict__ expo_b,
                                                     const double *__restrict__ scratch, int S, int32_t *__restrict__ err) {
    extern __shared__ uint8_t smem_dyn[];
    __shared__ Pipe pp;
    uint8_t *smem = align1024(smem_dyn);
    const HWork it = work[w0 + blockIdx.x];  // batch, 128-point tile, TN-function tile
    const int b = it.batch, m = s.sys.bmol[b];
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const SplitGeom G(P, N, S);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t tm = tc_setup(pp);
    const uint8_t *base = slices + sl_off[b];
    LoopArgs L;
    L.a0 = base + G.nA_block(0, 0) + (size_t)it.ti * 128 * 128;
    L.a_s = (size_t)G.n_kcN * G.P16 * 128;
    L.a_kc = (size_t)G.P16 * 128;
    L.b0 = base + G.nB_block(S, 0, 0) + (size_t)it.tj * TN * 128;
    L.b_s = (size_t)G.n_kcN * G.R16 * 128;
    L.b_kc = (size_t)G.R16 * 128;
    L.a_bytes = (uint32_t)min(128, G.P16 - it.ti * 128) * 128u;
    L.b_bytes = (uint32_t)min(TN, G.R16 - it.tj * TN) * 128u;
    // P' is zero for basis functions beyond tile J, so K stops at TN (J + 1)
    const int nk = ((it.tj + 1) * TN + 63) / 64;
    L.n_kc = nk < G.n_kcN ? nk : G.n_kcN;
    L.neg16 = 0;
    L.S = S;
    pipe_run<TN>(pp, smem, tm, L, err);
    if (!pp.abort) {
        const int q = it.ti * 128 + warp * 32 + lane;
        const bool row_ok = q < P;
        const int eq = row_ok ? expo_q[p0 + q] : -10000;
        const int eb = expo_b[b];
        const double *E = scratch + s.scr_off[b];
        const uint32_t tm_row = tm + ((uint32_t)(warp * 32) << 16);
        double part_hi = 0.0, part_lo = 0.0, part_lo2 = 0.0;
        for (int c0 = 0; c0 < TN; c0 += 16) {
            Parts16 v;
            combine16<TN>(tm_row, c0, S, v);
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const int j = it.tj * TN + c0 + jj;
                if (row_ok && j < N) {
                    const double f = E[(int64_t)j * Ppad + q];
                    part_hi = fma((double)v.hi[jj], f, part_hi);
                    part_lo = fma((double)v.lo[jj], f, part_lo);
                    part_lo2 = fma((double)v.lo2[jj], f, part_lo2);
                }
            }
        }
        if (row_ok && eq > -10000 && eb > -10000)
            atomicAdd(n_at(s, m, p0 + q), fma(part_hi, pow2(eq + eb - 48),
                                              fma(part_lo, pow2(eq + eb - 66), part_lo2 * pow2(eq + eb - 84))));
    }
    tc_teardown(tm);
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

}  // namespace

size_t split_smem_bytes(int S) { return pipe_smem_bytes(S); }

cudaError_t split_configure() {
    size_t bytes = 0;
    for (int S = 4; S <= NAO_SPLIT_MAX_SLICES; S++) bytes = split_smem_bytes(S) > bytes ? split_smem_bytes(S) : bytes;
    const void *fns[4] = {(const void *)h_tc_kernel<48>, (const void *)h_tc_kernel<32>, (const void *)n_tc_kernel<48>,
                          (const void *)n_tc_kernel<32>};
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
                        const int64_t *sl_off, const int32_t *expo, const int32_t *neg16, int S, int32_t *err,
                        cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    if (nao_split_tn(S) == 48)
        h_tc_kernel<48><<<n_work, 128, split_smem_bytes(S), st>>>(s, work, w0, slices, sl_off, expo, neg16, S, err);
    else
        h_tc_kernel<32><<<n_work, 128, split_smem_bytes(S), st>>>(s, work, w0, slices, sl_off, expo, neg16, S, err);
    return cudaGetLastError();
}

cudaError_t launch_slice_n(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_qt, const double *scratch,
                           uint8_t *slices, const int64_t *sl_off, int32_t *expo_q, int32_t *expo_b, int S,
                           cudaStream_t st) {
    if (b1 <= b0) return cudaSuccess;
    if (max_qt > 0) {
#define NAO_SLICE_NPHI(SS) \
    slice_nphi_kernel<SS><<<dim3(b1 - b0, max_qt), 128, 0, st>>>(s, b0, scratch, slices, sl_off, expo_q)
        NAO_SPLIT_DISPATCH(S, NAO_SLICE_NPHI)
#undef NAO_SLICE_NPHI
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
#define NAO_SLICE_NP(SS) slice_np_kernel<SS><<<b1 - b0, 256, 0, st>>>(s, b0, slices, sl_off, expo_b)
    NAO_SPLIT_DISPATCH(S, NAO_SLICE_NP)
#undef NAO_SLICE_NP
    return cudaGetLastError();
}

cudaError_t launch_n_tc(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                        const int64_t *sl_off, const int32_t *expo_q, const int32_t *expo_b, const double *scratch, int S,
                        int32_t *err, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    if (nao_split_tn(S) == 48)
        n_tc_kernel<48><<<n_work, 128, split_smem_bytes(S), st>>>(s, work, w0, slices, sl_off, expo_q, expo_b, scratch,
                                                                  S, err);
    else
        n_tc_kernel<32><<<n_work, 128, split_smem_bytes(S), st>>>(s, work, w0, slices, sl_off, expo_q, expo_b, scratch,
                                                                  S, err);
    return cudaGetLastError();
}

cudaError_t launch_wn_partial(const DevSystem &s, const DWork *work, int32_t w0, int32_t n_work, double *ne_part,
                              cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    wn_partial_kernel<<<n_work, 256, 0, st>>>(s, work, w0, ne_part);
    return cudaGetLastError();
}

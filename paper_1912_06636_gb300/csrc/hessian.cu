// Density Hessian on the FP64 and FP32 paths (Sec. 2: the six second derivatives of Eq. Density
// needed for forces and stresses, each a "straightforward extension" of the density).
//
// For symmetric P, differentiating n = sum_ij phi_i P_ij phi_j twice gives
//   d_a d_b n = 2 sum_ij P_ij (phi_i d_a d_b phi_j + d_a phi_i d_b phi_j),
// so per batch, with T = Phi P and T_a = (d_a Phi) P over the batch's reduced basis,
//   d_a d_b n_q = 2 sum_j (T_qj d_a d_b phi_qj + T_a,qj d_b phi_qj),
// and the same pass gives n_q = sum_j T_qj phi_qj and d_a n_q = 2 sum_j T_qj d_a phi_qj.
//
// Evaluation: one CTA per batch, one thread per (point, atom) as in the other evaluation
// kernels; phi = g(r) S_lm with g = R / r^l and S_lm = K Pi_l^m(z, r^2) {A_m, B_m}(x, y) (the
// solid-harmonic recurrence, carried with the first and second derivatives of Pi in z and r^2):
//   d_a phi     = g' (x_a / r) S + g d_a S,
//   d_a d_b phi = (g'' / r^2 - g' / r^3) x_a x_b S + (g' / r)(delta_ab S + x_b d_a S + x_a d_b S)
//                 + g d_a d_b S,
//   g' = R' / r^l - l R / r^(l+1),  g'' = R'' / r^l - 2 l R' / r^(l+1) + l (l+1) R / r^(l+2),
// with R' and R'' from the spline in s = ln(r / r0) / Delta (ds/dr = 1 / (r Delta),
// d^2s/dr^2 = -1 / (r^2 Delta)). Every batch's block of scratch holds, per reduced-basis row,
// 10 rows of Ppad points: phi, d/dx, d/dy, d/dz, xx, xy, xz, yy, yz, zz, in the path's type T
// (the values are computed in FP64 on both paths; the FP32 path rounds them once when storing).
// For the Pulay terms (LAP) the fifth row holds the Laplacian xx + yy + zz instead, summed in
// FP64 before the rounding (the three terms cancel where the Laplacian is small).
//
// Contraction: one CTA per 64-point density tile; for each 64-function tile J the four
// products Phi P, (d_x Phi) P, (d_y Phi) P, (d_z Phi) P over all of K in T (P read from its
// upper triangle, so the matrix used is exactly symmetric), then the epilogue above in T, the
// per-tile sums added in FP64. Every point is written once (no atomics).
#include <cmath>

#include "nao_internal.h"

namespace {

constexpr int HR = 10;       // rows per basis function in the Hessian scratch
constexpr int TQ = NAO_TILE; // 64 points per density tile
constexpr int TJ = 64;       // functions per tile
constexpr int KC = 8;        // K chunk of the contraction

__host__ __device__ constexpr double dfact_odd(int m) { return m <= 1 ? 1.0 : (2 * m - 1) * dfact_odd(m - 1); }

// (xx, xy, xz, yy, yz, zz)
__device__ __forceinline__ int pair_a(int k) { return k < 3 ? 0 : (k < 5 ? 1 : 2); }
__device__ __forceinline__ int pair_b(int k) { return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 2 : k == 3 ? 1 : 2; }

template <int LMAX, typename OutT, bool LAP>
__device__ __noinline__ void eval_group_hess(const DevSystem &s, const AtomGroup &ag, double x, double y, double z,
                                             double r2, double r, OutT *E, int64_t rs, int64_t cs, int q) {
    // radial coordinate (the radial part is taken at r0 for r < r0)
    const double rr = fmax(r, s.r0);
    const double sc = log(rr / s.r0) * s.inv_delta;
    int k = (int)floor(sc);
    k = k < 0 ? 0 : (k > s.n_rgrid - 2 ? s.n_rgrid - 2 : k);
    const double t = sc - (double)k;
    const double ds1 = s.inv_delta / rr, ds2 = -s.inv_delta / (rr * rr);
    const double ur = 1.0 / r;
    const double xa[3] = {x, y, z};

    // A_m + i B_m = (x + i y)^m
    double A[LMAX + 1], B[LMAX + 1];
    A[0] = 1.0;
    B[0] = 0.0;
#pragma unroll
    for (int m = 1; m <= LMAX; m++) {
        A[m] = x * A[m - 1] - y * B[m - 1];
        B[m] = x * B[m - 1] + y * A[m - 1];
    }
    // Pi_{l-1}^m (c) and Pi_{l-2}^m (p) with derivatives in z and q = r^2:
    // component 0 value, 1 d/dz, 2 d/dq, 3 d2/dz2, 4 d2/dzdq, 5 d2/dq2
    double Pc[6][LMAX + 1], Pp[6][LMAX + 1];
#pragma unroll
    for (int c = 0; c < 6; c++)
#pragma unroll
        for (int m = 0; m <= LMAX; m++) Pc[c][m] = Pp[c][m] = 0.0;
    int ri = ag.r0;
    const int re = ag.r0 + ag.nr;
    double rl = 1.0;  // r^l
#pragma unroll
    for (int l = 0; l <= LMAX; l++) {
        double S[2 * LMAX + 1], Sg[3][2 * LMAX + 1], Sh[6][2 * LMAX + 1];
#pragma unroll
        for (int m = 0; m <= l; m++) {
            double pv[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            if (m == l) {
                pv[0] = dfact_odd(m);
            } else if (m == l - 1) {
                pv[0] = (2 * m + 1) * z * Pc[0][m];
                pv[1] = (2 * m + 1) * Pc[0][m];
            } else {
                const double c1 = (double)(2 * l - 1) / (double)(l - m), c2 = (double)(l + m - 1) / (double)(l - m);
                pv[0] = c1 * z * Pc[0][m] - c2 * r2 * Pp[0][m];
                pv[1] = c1 * (Pc[0][m] + z * Pc[1][m]) - c2 * r2 * Pp[1][m];
                pv[2] = c1 * z * Pc[2][m] - c2 * (Pp[0][m] + r2 * Pp[2][m]);
                pv[3] = c1 * (2.0 * Pc[1][m] + z * Pc[3][m]) - c2 * r2 * Pp[3][m];
                pv[4] = c1 * (Pc[2][m] + z * Pc[4][m]) - c2 * (Pp[1][m] + r2 * Pp[4][m]);
                pv[5] = c1 * z * Pc[5][m] - c2 * (2.0 * Pp[2][m] + r2 * Pp[5][m]);
            }
#pragma unroll
            for (int c = 0; c < 6; c++) {
                Pp[c][m] = Pc[c][m];
                Pc[c][m] = pv[c];
            }
            // P(x, y, z) = Pi(z, q(x, y, z)) and its derivatives
            const double P0 = pv[0];
            const double Pd[3] = {2.0 * x * pv[2], 2.0 * y * pv[2], pv[1] + 2.0 * z * pv[2]};
            const double Pdd[6] = {2.0 * pv[2] + 4.0 * x * x * pv[5],                       // xx
                                   4.0 * x * y * pv[5],                                       // xy
                                   2.0 * x * (pv[4] + 2.0 * z * pv[5]),                       // xz
                                   2.0 * pv[2] + 4.0 * y * y * pv[5],                       // yy
                                   2.0 * y * (pv[4] + 2.0 * z * pv[5]),                       // yz
                                   pv[3] + 4.0 * z * pv[4] + 2.0 * pv[2] + 4.0 * z * z * pv[5]};  // zz
            const double kn = s.knorm[l][m];
            // the x, y factor C and its derivatives (d/dz = 0): m = 0: C = 1; m > 0: C = A_m or B_m
            for (int part = 0; part < (m == 0 ? 1 : 2); part++) {
                double C = 1.0, Cd[3] = {0.0, 0.0, 0.0}, Cdd[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                const double fm = (double)m, fmm = (double)(m * (m - 1));
                if (m > 0 && part == 0) {  // A_m: d/dx = m A_{m-1}, d/dy = -m B_{m-1}
                    C = A[m];
                    Cd[0] = fm * A[m - 1];
                    Cd[1] = -fm * B[m - 1];
                    if (m >= 2) {
                        Cdd[0] = fmm * A[m - 2];
                        Cdd[1] = -fmm * B[m - 2];
                        Cdd[3] = -fmm * A[m - 2];
                    }
                } else if (m > 0) {        // B_m: d/dx = m B_{m-1}, d/dy = m A_{m-1}
                    C = B[m];
                    Cd[0] = fm * B[m - 1];
                    Cd[1] = fm * A[m - 1];
                    if (m >= 2) {
                        Cdd[0] = fmm * B[m - 2];
                        Cdd[1] = fmm * A[m - 2];
                        Cdd[3] = -fmm * B[m - 2];
                    }
                }
                const int idx = m == 0 ? l : (part == 0 ? l + m : l - m);
                S[idx] = kn * P0 * C;
#pragma unroll
                for (int a = 0; a < 3; a++) Sg[a][idx] = kn * (Pd[a] * C + P0 * Cd[a]);
#pragma unroll
                for (int kk = 0; kk < 6; kk++) {
                    const int a = pair_a(kk), b = pair_b(kk);
                    Sh[kk][idx] = kn * (Pdd[kk] * C + Pd[a] * Cd[b] + Pd[b] * Cd[a] + P0 * Cdd[kk]);
                }
            }
        }
        // the atom's radial functions of this l
        for (; ri < re; ri++) {
            const RfnEntry e = s.rfn[ri];
            if (e.l != l) break;
            double g = 0.0, G1 = 0.0, Q = 0.0;  // g, g'/r, g''/r^2 - g'/r^3
            if (r < s.fn_rc[e.fn]) {
                const double *cf = s.coef + ((size_t)e.fn * (s.n_rgrid - 1) + k) * 4;
                const double R = ((cf[3] * t + cf[2]) * t + cf[1]) * t + cf[0];
                const double Rs = (3.0 * cf[3] * t + 2.0 * cf[2]) * t + cf[1];
                const double Rss = 6.0 * cf[3] * t + 2.0 * cf[2];
                const double R1 = Rs * ds1, R2 = Rss * ds1 * ds1 + Rs * ds2;
                const double fl = (double)l;
                g = R / rl;
                const double g1 = R1 / rl - fl * R / (rl * r);
                const double g2 = R2 / rl - 2.0 * fl * R1 / (rl * r) + fl * (fl + 1.0) * R / (rl * r * r);
                G1 = g1 * ur;
                Q = g2 * ur * ur - g1 * ur * ur * ur;
            }
            for (int mm = 0; mm < 2 * l + 1; mm++) {
                OutT *row = E + (int64_t)(e.pos + mm) * rs + q;
                const double Sv = S[mm];
                row[0] = OutT(g * Sv);
#pragma unroll
                for (int a = 0; a < 3; a++) row[(1 + a) * cs] = OutT(G1 * xa[a] * Sv + g * Sg[a][mm]);
                double lap = 0.0;
#pragma unroll
                for (int kk = 0; kk < 6; kk++) {
                    const int a = pair_a(kk), b = pair_b(kk);
                    const double dab = a == b ? 1.0 : 0.0;
                    const double v = Q * xa[a] * xa[b] * Sv + G1 * (dab * Sv + xa[b] * Sg[a][mm] + xa[a] * Sg[b][mm]) +
                                     g * Sh[kk][mm];
                    if (LAP) {
                        if (a == b) lap += v;  // xx + yy + zz, in that order
                    } else {
                        row[(4 + kk) * cs] = OutT(v);
                    }
                }
                if (LAP) row[4 * cs] = OutT(lap);
            }
        }
        rl *= r;
    }
}

template <typename OutT, bool LAP>
__global__ void __launch_bounds__(256) eval_hess_kernel(DevSystem s, int32_t b0, OutT *__restrict__ scratch,
                                                       const int64_t *__restrict__ hoff) {
    const int b = b0 + blockIdx.x;
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int g0 = s.agrp_off[b], ng = s.agrp_off[b + 1] - g0;
    OutT *E = scratch + hoff[b];
    const int64_t rs = (int64_t)HR * Ppad, cs = Ppad;
    for (int idx = threadIdx.x; idx < ng * Ppad; idx += blockDim.x) {
        const int gl = idx / Ppad, q = idx - gl * Ppad;
        const AtomGroup ag = s.agrp[g0 + gl];
        if (q >= P) {  // padding points: zero rows
            for (int ri = ag.r0; ri < ag.r0 + ag.nr; ri++) {
                const RfnEntry e = s.rfn[ri];
                for (int mm = 0; mm < 2 * e.l + 1; mm++)
                    for (int c = 0; c < HR; c++) E[(int64_t)(e.pos + mm) * rs + c * cs + q] = OutT(0);
            }
            continue;
        }
        const int p = p0 + q;
        const double dx = s.px[p] - s.atom_xyz[3 * ag.atom], dy = s.py[p] - s.atom_xyz[3 * ag.atom + 1],
                     dz = s.pz[p] - s.atom_xyz[3 * ag.atom + 2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double r = sqrt(r2);
        switch (ag.lmax) {
            case 0: eval_group_hess<0, OutT, LAP>(s, ag, dx, dy, dz, r2, r, E, rs, cs, q); break;
            case 1: eval_group_hess<1, OutT, LAP>(s, ag, dx, dy, dz, r2, r, E, rs, cs, q); break;
            case 2: eval_group_hess<2, OutT, LAP>(s, ag, dx, dy, dz, r2, r, E, rs, cs, q); break;
            case 3: eval_group_hess<3, OutT, LAP>(s, ag, dx, dy, dz, r2, r, E, rs, cs, q); break;
            case 4: eval_group_hess<4, OutT, LAP>(s, ag, dx, dy, dz, r2, r, E, rs, cs, q); break;
            case 5: eval_group_hess<5, OutT, LAP>(s, ag, dx, dy, dz, r2, r, E, rs, cs, q); break;
            default: eval_group_hess<6, OutT, LAP>(s, ag, dx, dy, dz, r2, r, E, rs, cs, q); break;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) density_hess_kernel(DevSystem s, const DWork *__restrict__ work, int32_t w0,
                                                          const T *__restrict__ scratch,
                                                          const int64_t *__restrict__ hoff, double *__restrict__ hess,
                                                          double *__restrict__ ne_part) {
    __shared__ __align__(16) T As[4][KC][TQ];  // phi, d/dx, d/dy, d/dz of rows i, at the tile's points
    __shared__ __align__(16) T Bs[KC][TJ];     // P[rel_i][rel_j]
    __shared__ double acc_n[TQ], acc_g[3][TQ], acc_h[6][TQ];
    __shared__ double red[8];
    const DWork it = work[w0 + blockIdx.x];
    const int b = it.batch, m = s.sys.bmol[b];
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const int q0 = it.tp * TQ;
    const T *E = scratch + hoff[b];
    const int64_t ld = (int64_t)HR * Ppad;
    const int32_t *rel = s.rel_idx + s.rel_off[b];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < TQ) {
        acc_n[tid] = 0.0;
        for (int c = 0; c < 3; c++) acc_g[c][tid] = 0.0;
        for (int c = 0; c < 6; c++) acc_h[c][tid] = 0.0;
    }
    const int nt = (N + TJ - 1) / TJ;
    for (int tj = 0; tj < nt; tj++) {
        T Tm[4][4][4];
#pragma unroll
        for (int c = 0; c < 4; c++)
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int d = 0; d < 4; d++) Tm[c][a][d] = T(0);
        for (int i0 = 0; i0 < N; i0 += KC) {
            __syncthreads();
            for (int u = tid; u < 4 * KC * TQ; u += blockDim.x) {
                const int c = u / (KC * TQ), kk = (u / TQ) % KC, qq = u % TQ;
                const int i = i0 + kk, q = q0 + qq;
                As[c][kk][qq] = (i < N && q < Ppad) ? E[(int64_t)i * ld + (int64_t)c * Ppad + q] : T(0);
            }
            for (int u = tid; u < KC * TJ; u += blockDim.x) {
                const int kk = u / TJ, jj = u % TJ;
                const int i = i0 + kk, j = tj * TJ + jj;
                double pv = 0.0;
                if (i < N && j < N) {
                    int64_t gi = rel[i], gj = rel[j];
                    if (gi > gj) { const int64_t tt = gi; gi = gj; gj = tt; }
                    pv = p_elem(s, m, gi, gj);
                }
                Bs[kk][jj] = T(pv);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KC; kk++) {
                T rb[4];
#pragma unroll
                for (int d = 0; d < 4; d++) rb[d] = Bs[kk][tx * 4 + d];
#pragma unroll
                for (int c = 0; c < 4; c++)
#pragma unroll
                    for (int a = 0; a < 4; a++) {
                        const T ra = As[c][kk][ty * 4 + a];
#pragma unroll
                        for (int d = 0; d < 4; d++) Tm[c][a][d] = fma(ra, rb[d], Tm[c][a][d]);
                    }
            }
        }
        // epilogue: rows q = q0 + ty*4 + a, columns j = tj*64 + tx*4 + d
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int q = q0 + ty * 4 + a;
            T pn = T(0), pg[3] = {T(0), T(0), T(0)}, ph[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int d = 0; d < 4; d++) {
                const int j = tj * TJ + tx * 4 + d;
                if (j < N && q < Ppad) {
                    const T *f = E + (int64_t)j * ld + q;
                    T fv[HR];
#pragma unroll
                    for (int c = 0; c < HR; c++) fv[c] = f[(int64_t)c * Ppad];
                    pn = fma(Tm[0][a][d], fv[0], pn);
#pragma unroll
                    for (int c = 0; c < 3; c++) pg[c] = fma(Tm[0][a][d], fv[1 + c], pg[c]);
#pragma unroll
                    for (int kk = 0; kk < 6; kk++)
                        ph[kk] = fma(Tm[1 + pair_a(kk)][a][d], fv[1 + pair_b(kk)], fma(Tm[0][a][d], fv[4 + kk], ph[kk]));
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                pn += __shfl_xor_sync(0xffffffffu, pn, o);
#pragma unroll
                for (int c = 0; c < 3; c++) pg[c] += __shfl_xor_sync(0xffffffffu, pg[c], o);
#pragma unroll
                for (int kk = 0; kk < 6; kk++) ph[kk] += __shfl_xor_sync(0xffffffffu, ph[kk], o);
            }
            if (tx == 0) {
                acc_n[ty * 4 + a] += (double)pn;
#pragma unroll
                for (int c = 0; c < 3; c++) acc_g[c][ty * 4 + a] += 2.0 * (double)pg[c];
#pragma unroll
                for (int kk = 0; kk < 6; kk++) acc_h[kk][ty * 4 + a] += 2.0 * (double)ph[kk];
            }
        }
    }
    __syncthreads();
    double wn = 0.0;
    if (tid < TQ) {
        const int q = q0 + tid;
        if (q < P) {
            const int p = p0 + q;
            *n_at(s, m, p) = acc_n[tid];
            for (int c = 0; c < 3; c++) *gn_at(s, m, p, c) = acc_g[c][tid];
            const int64_t np = s.sys.np[m], o = s.perm[p] - s.sys.poff[m];
            for (int c = 0; c < 6; c++) hess[(int64_t)c * np + o] = acc_h[c][tid];
            wn = s.pw[p] * acc_n[tid];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) wn += __shfl_xor_sync(0xffffffffu, wn, o);
    if ((tid & 31) == 0) red[tid >> 5] = wn;
    __syncthreads();
    if (tid == 0) {
        double tsum = 0.0;
        for (int w = 0; w < 8; w++) tsum += red[w];
        ne_part[w0 + blockIdx.x] = tsum;
    }
}

}  // namespace

cudaError_t launch_eval_hess(const DevSystem &s, int32_t b0, int32_t b1, void *scratch, bool fp32, bool lap,
                             const int64_t *hoff, cudaStream_t st) {
    if (b1 <= b0) return cudaSuccess;
    const int n = b1 - b0;
    if (fp32 && lap) eval_hess_kernel<float, true><<<n, 256, 0, st>>>(s, b0, static_cast<float *>(scratch), hoff);
    else if (fp32) eval_hess_kernel<float, false><<<n, 256, 0, st>>>(s, b0, static_cast<float *>(scratch), hoff);
    else if (lap) eval_hess_kernel<double, true><<<n, 256, 0, st>>>(s, b0, static_cast<double *>(scratch), hoff);
    else eval_hess_kernel<double, false><<<n, 256, 0, st>>>(s, b0, static_cast<double *>(scratch), hoff);
    return cudaGetLastError();
}

cudaError_t launch_density_hess(const DevSystem &s, const DWork *work, int32_t w0, int32_t n_work, const void *scratch,
                                bool fp32, const int64_t *hoff, double *hess, double *ne_part, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    if (fp32)
        density_hess_kernel<float><<<n_work, 256, 0, st>>>(s, work, w0, static_cast<const float *>(scratch), hoff, hess,
                                                            ne_part);
    else
        density_hess_kernel<double><<<n_work, 256, 0, st>>>(s, work, w0, static_cast<const double *>(scratch), hoff,
                                                             hess, ne_part);
    return cudaGetLastError();
}

// Local Pulay force terms on the FP64 and FP32 paths (Sec. 2, the local parts of the Pulay forces,
//     F_at = -2 sum_ij int [grad_at phi_i] n_ij h_KS phi_j + 2 sum_ij int [grad_at phi_i] q_ij phi_j,
// q the energy-weighted density matrix), assembled, as the paper describes for forces, from
// matrix elements with basis-function indices first (Sec. "Density and Density Derivatives"):
//     M^c_ij = sum_p w_p d_c phi_i (h phi_j),  h phi_j = -1/2 lap phi_j + v phi_j,
//     S^c_ij = sum_p w_p d_c phi_i phi_j,                       c = x, y, z,
// then, since grad_at phi_i = -grad phi_i for a function on atom at,
//     F_at,c = 2 sum_{i on at} sum_j (n_ij M^c_ij - q_ij S^c_ij).
// The batches' basis functions come from the density Hessian's evaluation (10 rows per function:
// phi, grad phi and, in place of the six second derivatives, lap = xx + yy + zz summed in FP64).
// One CTA per 64 x 64 tile pair (I, J) of a batch (all pairs: the matrices are not symmetric); per 8-point K chunk the CTA
// stages w d_c phi_i (three components) and h phi_j, phi_j, and accumulates the six products in
// the path's type T (the evaluation is FP64 on both paths, stored in T; on the FP32 path each
// 8-point chunk's sums are added into compensated (hi, lo) pairs, in two passes of three
// products); FP64 atomics add each tile into the global matrices.
#include <type_traits>

#include "nao_internal.h"

namespace {

constexpr int HR = 10;  // rows per basis function in the Hessian evaluation
constexpr int TT = 64;  // tile edge (functions)
constexpr int KC = 8;   // points per K chunk

// (hi, lo) += x with Knuth's TwoSum (exact transformation of hi + x): the FP32 path's running
// sums over the chunks, so that only each 8-point chunk is summed in plain FP32.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
    const float t = __fadd_rn(hi, x);
    const float bb = __fsub_rn(t, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
    hi = t;
}

// NU = 2: both products (h phi_j and phi_j) in one pass (FP64); NU = 1: the product u0 only
// (FP32: two passes, which leaves registers for the compensated sums).
template <typename T, int NU>
__global__ void __launch_bounds__(256) pulay_kernel(DevSystem s, const HWork *__restrict__ work, int32_t w0,
                                                   const T *__restrict__ scratch, const int64_t *__restrict__ hoff,
                                                   double *__restrict__ M, double *__restrict__ Sm, int64_t nb, int u0) {
    constexpr bool F32 = std::is_same<T, float>::value;
    __shared__ __align__(16) T As[3][KC][TT];  // w_q d_c phi_i(q)
    __shared__ __align__(16) T Bs[NU][KC][TT];  // h phi_j(q) (u = 0), phi_j(q) (u = 1)
    const HWork it = work[w0 + blockIdx.x];
    const int b = it.batch, m = s.sys.bmol[b];
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const T *E = scratch + hoff[b];
    const int64_t ld = (int64_t)HR * Ppad;
    const int32_t *rel = s.rel_idx + s.rel_off[b];
    const int i0 = it.ti * TT, j0 = it.tj * TT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T acc[3][NU][4][4];
    float hi[3][NU][4][4], lo[3][NU][4][4];  // FP32 only (unused, and removed, for FP64)
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
        for (int u = 0; u < NU; u++)
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int d = 0; d < 4; d++) {
                    acc[c][u][a][d] = T(0);
                    hi[c][u][a][d] = lo[c][u][a][d] = 0.0f;
                }
    for (int q0 = 0; q0 < P; q0 += KC) {
        __syncthreads();
        for (int u = tid; u < 3 * KC * TT; u += blockDim.x) {
            const int c = u / (KC * TT), kk = (u / TT) % KC, ii = u % TT;
            const int i = i0 + ii, q = q0 + kk;
            As[c][kk][ii] = (i < N && q < P) ? T(s.pw[p0 + q] * (double)E[(int64_t)i * ld + (int64_t)(1 + c) * Ppad + q]) : T(0);
        }
        for (int u = tid; u < KC * TT; u += blockDim.x) {
            const int kk = u / TT, jj = u % TT;
            const int j = j0 + jj, q = q0 + kk;
            double hphi = 0.0, f = 0.0;
            if (j < N && q < P) {
                const T *row = E + (int64_t)j * ld + q;
                f = (double)row[0];
                if (NU == 2 || u0 == 0) {
                    const double lap = (double)row[4 * (int64_t)Ppad];  // the evaluation's Laplacian row
                    hphi = -0.5 * lap + v_at(s, m, p0 + q) * f;
                }
            }
            if (NU == 2) {
                Bs[0][kk][jj] = T(hphi);
                Bs[NU - 1][kk][jj] = T(f);
            } else {
                Bs[0][kk][jj] = T(u0 == 0 ? hphi : f);
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KC; kk++) {
            T rb[NU][4];
#pragma unroll
            for (int u = 0; u < NU; u++)
#pragma unroll
                for (int d = 0; d < 4; d++) rb[u][d] = Bs[u][kk][tx * 4 + d];
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int a = 0; a < 4; a++) {
                    const T ra = As[c][kk][ty * 4 + a];
#pragma unroll
                    for (int u = 0; u < NU; u++)
#pragma unroll
                        for (int d = 0; d < 4; d++) acc[c][u][a][d] = fma(ra, rb[u][d], acc[c][u][a][d]);
                }
        }
        if constexpr (F32) {
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int u = 0; u < NU; u++)
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int d = 0; d < 4; d++) {
                            two_sum_acc(hi[c][u][a][d], lo[c][u][a][d], (float)acc[c][u][a][d]);
                            acc[c][u][a][d] = T(0);
                        }
        }
    }
    const int64_t nn = nb * nb;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int i = i0 + ty * 4 + a;
        if (i >= N) continue;
        const int64_t gi = rel[i];
#pragma unroll
        for (int d = 0; d < 4; d++) {
            const int j = j0 + tx * 4 + d;
            if (j >= N) continue;
            const int64_t e = gi * nb + rel[j];
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int u = 0; u < NU; u++) {
                    const double v = F32 ? (double)hi[c][u][a][d] + (double)lo[c][u][a][d] : (double)acc[c][u][a][d];
                    atomicAdd(((NU == 2 ? u : u0) == 0 ? M : Sm) + c * nn + e, v);
                }
        }
    }
}

// One CTA per atom: F[3 a + c] = 2 sum_{i on a} sum_j (n_ij M^c_ij - q_ij S^c_ij).
__global__ void __launch_bounds__(256) pulay_force_kernel(const double *__restrict__ nmat, const double *__restrict__ qmat,
                                                         const double *__restrict__ M, const double *__restrict__ Sm,
                                                         const int64_t *__restrict__ atom_basis, int64_t nb,
                                                         double *__restrict__ F) {
    __shared__ double red[3][8];
    const int a = blockIdx.x;
    const int64_t i0 = atom_basis[a], i1 = atom_basis[a + 1], nn = nb * nb;
    double part[3] = {0.0, 0.0, 0.0};
    for (int64_t e = i0 * nb + threadIdx.x; e < i1 * nb; e += blockDim.x) {
        const double n = nmat[e], q = qmat[e];
#pragma unroll
        for (int c = 0; c < 3; c++) part[c] = fma(n, M[c * nn + e], fma(-q, Sm[c * nn + e], part[c]));
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part[c] += __shfl_xor_sync(0xffffffffu, part[c], o);
        if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = part[c];
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += red[threadIdx.x][w];
        F[3 * a + threadIdx.x] = 2.0 * t;
    }
}

}  // namespace

cudaError_t launch_pulay(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const void *scratch, bool fp32,
                         const int64_t *hoff, double *M, double *S, int64_t nb, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    if (fp32) {
        for (int u0 = 0; u0 < 2; u0++) {
            pulay_kernel<float, 1><<<n_work, 256, 0, st>>>(s, work, w0, static_cast<const float *>(scratch), hoff, M, S, nb, u0);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    } else {
        pulay_kernel<double, 2><<<n_work, 256, 0, st>>>(s, work, w0, static_cast<const double *>(scratch), hoff, M, S, nb, 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_pulay_forces(const double *nmat, const double *qmat, const double *M, const double *S,
                                const int64_t *atom_basis, int32_t n_atoms, int64_t nb, double *F, cudaStream_t st) {
    if (n_atoms <= 0) return cudaSuccess;
    pulay_force_kernel<<<n_atoms, 256, 0, st>>>(nmat, qmat, M, S, atom_basis, nb, F);
    return cudaGetLastError();
}

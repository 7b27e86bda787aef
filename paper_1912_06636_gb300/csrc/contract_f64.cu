// FP64 contractions on the CUDA cores.
//
// Hamiltonian (Eq. batch_matrix_mult with K and L stacked over the potential and the three
// gradient components): for batch B with reduced basis of size N and points padded to Ppad,
// the evaluated block E (N rows x 4 Ppad columns: phi | d/dx | d/dy | d/dz) gives
//   h[B]_ij = sum_k E_ik d_k E_jk,  d_k = w_q v_q (phi part) or w_q / 2 (gradient parts),
// computed for upper-triangular 64 x 64 tile pairs (I <= J) only and added into the global
// H[rel_i][rel_j] with FP64 atomics (the indexing step, Sec. 3.4 (ii)); a final pass copies
// the upper triangle onto the lower one, so H is exactly symmetric.
//
// Density (Eq. Density, restricted to nnz(B)): n_q = sum_ij phi_iq P_ij phi_jq, evaluated per
// 64-point tile as sum over tile pairs I <= J of c_IJ sum_{i in I, j in J} phi_iq P_ij phi_jq
// with c_II = 1 and c_IJ = 2 (I < J), which reads only P's upper triangle.
#include "nao_internal.h"

namespace {

constexpr int T = NAO_TILE;  // 64
constexpr int KC = 16;       // K chunk

__global__ void __launch_bounds__(256) h_f64_kernel(DevSystem s, const HWork *__restrict__ work,
                                                   const double *__restrict__ scratch, const double *__restrict__ v,
                                                   uint32_t terms, double *__restrict__ H) {
    extern __shared__ double dyn[];
    __shared__ double As[KC][T];
    __shared__ double Bs[KC][T];
    const HWork it = work[blockIdx.x];
    const int b = it.batch;
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const int64_t ld = 4 * (int64_t)Ppad;
    const double *E = scratch + s.scr_off[b];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

    double *dv = dyn, *dk = dyn + Ppad;  // weights of the potential and kinetic parts
    for (int q = tid; q < Ppad; q += blockDim.x) {
        const double w = q < P ? s.pw[p0 + q] : 0.0;
        const double vv = (q < P && v) ? v[s.perm[p0 + q]] : 1.0;
        dv[q] = (terms & NAO_TERM_POTENTIAL) ? w * vv : 0.0;
        dk[q] = (terms & NAO_TERM_KINETIC) ? 0.5 * w : 0.0;
    }

    const int i0 = it.ti * T, j0 = it.tj * T;
    const int lrow = tid >> 2, lk = (tid & 3) * 4;
    const bool arow_ok = i0 + lrow < N, brow_ok = j0 + lrow < N;
    const double *Arow = E + (int64_t)(i0 + lrow) * ld + lk;
    const double *Brow = E + (int64_t)(j0 + lrow) * ld + lk;

    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[a][c] = 0.0;

    __syncthreads();
    const int K = 4 * Ppad;
    for (int k0 = 0; k0 < K; k0 += KC) {
        const int comp = k0 / Ppad, qk = k0 - comp * Ppad + lk;
        const double *dw = comp == 0 ? dv : dk;
        double2 a01 = make_double2(0.0, 0.0), a23 = a01, b01 = a01, b23 = a01;
        if (arow_ok) {
            a01 = *reinterpret_cast<const double2 *>(Arow + k0);
            a23 = *reinterpret_cast<const double2 *>(Arow + k0 + 2);
        }
        if (brow_ok) {
            b01 = *reinterpret_cast<const double2 *>(Brow + k0);
            b23 = *reinterpret_cast<const double2 *>(Brow + k0 + 2);
        }
        As[lk + 0][lrow] = a01.x;
        As[lk + 1][lrow] = a01.y;
        As[lk + 2][lrow] = a23.x;
        As[lk + 3][lrow] = a23.y;
        Bs[lk + 0][lrow] = b01.x * dw[qk + 0];
        Bs[lk + 1][lrow] = b01.y * dw[qk + 1];
        Bs[lk + 2][lrow] = b23.x * dw[qk + 2];
        Bs[lk + 3][lrow] = b23.y * dw[qk + 3];
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KC; kk++) {
            double ra[4], rb[4];
#pragma unroll
            for (int a = 0; a < 4; a++) ra[a] = As[kk][ty + 16 * a];
#pragma unroll
            for (int c = 0; c < 4; c++) rb[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int c = 0; c < 4; c++) acc[a][c] = fma(ra[a], rb[c], acc[a][c]);
        }
        __syncthreads();
    }

    const int32_t *rel = s.rel_idx + s.rel_off[b];
    const bool diag = it.ti == it.tj;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int i = i0 + ty + 16 * a;
        if (i >= N) continue;
        const int64_t gi = rel[i];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int j = j0 + tx + 16 * c;
            if (j >= N || (diag && j < i)) continue;
            atomicAdd(H + gi * s.nb + rel[j], acc[a][c]);
        }
    }
}

// Copy the upper triangle onto the lower one through 32 x 32 shared-memory tiles.
__global__ void mirror_kernel(double *__restrict__ H, int64_t nb) {
    __shared__ double tile[32][33];
    const int bx = blockIdx.x, by = blockIdx.y;  // source tile (row block by, column block bx), by <= bx
    if (by > bx) return;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += blockDim.y) {
        const int64_t row = (int64_t)by * 32 + r, col = (int64_t)bx * 32 + tx;
        tile[r][tx] = (row < nb && col < nb) ? H[row * nb + col] : 0.0;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += blockDim.y) {
        const int64_t row = (int64_t)bx * 32 + r, col = (int64_t)by * 32 + tx;  // destination, lower part
        if (row < nb && col < nb && row > col) H[row * nb + col] = tile[tx][r];
    }
}

__global__ void __launch_bounds__(256) density_f64_kernel(DevSystem s, const DWork *__restrict__ work, int32_t w0,
                                                         const double *__restrict__ scratch,
                                                         const double *__restrict__ Pm, double *__restrict__ nout,
                                                         double *__restrict__ ne_part) {
    __shared__ double As[KC][T];  // phi[i][q]
    __shared__ double Bs[KC][T];  // c_IJ P[rel_i][rel_j]
    __shared__ double nacc[T];
    __shared__ double red[8];
    const DWork it = work[w0 + blockIdx.x];
    const int b = it.batch;
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const int q0 = it.tp * T;
    const double *E = scratch + s.scr_off[b];  // phi only: row stride Ppad
    const int32_t *rel = s.rel_idx + s.rel_off[b];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int nt = (N + T - 1) / T;
    if (tid < T) nacc[tid] = 0.0;

    const int lk = tid >> 4, lc = (tid & 15) * 4;  // loader: row k of the chunk, 4 columns
    for (int tj = 0; tj < nt; tj++) {
        double acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[a][c] = 0.0;
        for (int ti = 0; ti <= tj; ti++) {
            const double scale = ti < tj ? 2.0 : 1.0;
            for (int k0 = 0; k0 < T; k0 += KC) {
                const int i = ti * T + k0 + lk;
                // phi tile: 4 consecutive points of row i
                double2 f01 = make_double2(0.0, 0.0), f23 = f01;
                if (i < N && q0 + lc < Ppad) {
                    const double *src = E + (int64_t)i * Ppad + q0 + lc;
                    f01 = *reinterpret_cast<const double2 *>(src);
                    f23 = *reinterpret_cast<const double2 *>(src + 2);
                }
                As[lk][lc + 0] = f01.x;
                As[lk][lc + 1] = f01.y;
                As[lk][lc + 2] = f23.x;
                As[lk][lc + 3] = f23.y;
                // P tile: row rel_i, 4 columns rel_j (upper triangle only)
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int j = tj * T + lc + u;
                    double pv = 0.0;
                    if (i < N && j < N) {
                        int64_t gi = rel[i], gj = rel[j];
                        if (gi > gj) { const int64_t t = gi; gi = gj; gj = t; }
                        pv = scale * Pm[gi * s.nb + gj];
                    }
                    Bs[lk][lc + u] = pv;
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < KC; kk++) {
                    double ra[4], rb[4];
#pragma unroll
                    for (int a = 0; a < 4; a++) ra[a] = As[kk][ty + 16 * a];
#pragma unroll
                    for (int c = 0; c < 4; c++) rb[c] = Bs[kk][tx + 16 * c];
#pragma unroll
                    for (int a = 0; a < 4; a++)
#pragma unroll
                        for (int c = 0; c < 4; c++) acc[a][c] = fma(ra[a], rb[c], acc[a][c]);
                }
                __syncthreads();
            }
        }
        // n_q += sum_{j in J} T_qj phi_jq
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int q = q0 + ty + 16 * a;
            double part = 0.0;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int j = tj * T + tx + 16 * c;
                const double f = (j < N && q < Ppad) ? E[(int64_t)j * Ppad + q] : 0.0;
                part = fma(acc[a][c], f, part);
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (tx == 0) nacc[ty + 16 * a] += part;
        }
        __syncthreads();
    }
    __syncthreads();
    double wn = 0.0;
    if (tid < T) {
        const int q = q0 + tid;
        if (q < P) {
            const double nv = nacc[tid];
            nout[s.perm[p0 + q]] = nv;
            wn = s.pw[p0 + q] * nv;
        }
    }
    // fixed-order block sum of w n over the tile
    for (int o = 16; o > 0; o >>= 1) wn += __shfl_xor_sync(0xffffffffu, wn, o);
    if ((tid & 31) == 0) red[tid >> 5] = wn;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; w++) t += red[w];
        ne_part[w0 + blockIdx.x] = t;
    }
}

// Deterministic single-CTA sum (fixed assignment and fixed tree order).
__global__ void __launch_bounds__(1024) reduce_sum_kernel(const double *__restrict__ part, int64_t n,
                                                         double *__restrict__ out) {
    __shared__ double red[32];
    double t = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        t = red[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) out[0] = t;
    }
}

}  // namespace

cudaError_t launch_h_f64(const DevSystem &s, const HWork *work, int32_t n_work, const double *scratch,
                         const double *v, uint32_t terms, double *H, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    const size_t smem = 2 * sizeof(double) * NAO_MAX_BATCH;
    h_f64_kernel<<<n_work, 256, smem, st>>>(s, work, scratch, v, terms, H);
    return cudaGetLastError();
}

cudaError_t launch_mirror(double *H, int64_t nb, cudaStream_t st) {
    const unsigned g = (unsigned)((nb + 31) / 32);
    if (g == 0) return cudaSuccess;
    mirror_kernel<<<dim3(g, g), dim3(32, 8), 0, st>>>(H, nb);
    return cudaGetLastError();
}

cudaError_t launch_density_f64(const DevSystem &s, const DWork *work, int32_t w0, int32_t n_work,
                               const double *scratch, const double *P, double *n, double *ne_part, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    density_f64_kernel<<<n_work, 256, 0, st>>>(s, work, w0, scratch, P, n, ne_part);
    return cudaGetLastError();
}

cudaError_t launch_reduce_sum(const double *part, int64_t n, double *out, cudaStream_t st) {
    reduce_sum_kernel<<<1, 1024, 0, st>>>(part, n, out);
    return cudaGetLastError();
}

// Batch contractions on the CUDA cores, in FP64 or FP32 (T).
//
// Hamiltonian (Eq. batch_matrix_mult with K and L stacked over the potential and the three
// gradient components): for batch B with reduced basis of size N and points padded to Ppad,
// the evaluated block E (N rows x 4 Ppad columns: phi | d/dx | d/dy | d/dz) gives
//   h[B]_ij = sum_k E_ik d_k E_jk,  d_k = w_q v_q (phi part) or w_q / 2 (gradient parts),
// computed for upper-triangular 64 x 64 tile pairs (I <= J) only and added into the global
// H[rel_i][rel_j] with FP64 atomics (the indexing step of Sec. 3.4 (ii)); a final pass
// copies the upper triangle onto the lower one, so H is exactly symmetric.
//
// Density (Eq. Density restricted to nnz(B)): n_q = sum_ij phi_iq P_ij phi_jq, evaluated per
// 64-point tile as the sum over tile pairs I <= J of c_IJ sum_{i in I, j in J} phi_iq P_ij phi_jq
// with c_II = 1 and c_IJ = 2 (I < J), which reads only P's upper triangle.
//
// FP32: products accumulate in FP32 over chunks of 32 terms; each chunk sum is folded into an
// FP32 (hi, lo) pair with Knuth's TwoSum, and hi + lo is widened to FP64 for the scatter.
// FP64 work of any kind is ~60x slower than FP32 on this GPU, which rules out an FP64
// accumulator per chunk.
#include "nao_internal.h"

namespace {

constexpr int T_ = NAO_TILE;  // 64

template <typename T> struct Cfg;
template <> struct Cfg<double> { static constexpr int KC = 16; };
template <> struct Cfg<float> { static constexpr int KC = 32; };

__device__ __forceinline__ void load_vec(const double *p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void load_vec(const float *p, float (&v)[8]) {
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void lds4(const double *p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void lds4(const float *p, float (&v)[4]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

// (hi, lo) += x with Knuth's TwoSum (exact transformation of hi + x).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// 4 x 4 block accumulator: FP64 accumulates directly; FP32 keeps a chunk sum and a (hi, lo) pair.
template <typename T>
struct Block {
    T c[4][4];
    T hi[4][4], lo[4][4];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) c[a][b] = hi[a][b] = lo[a][b] = T(0);
    }
    __device__ __forceinline__ void fold() {
        if constexpr (std::is_same<T, float>::value) {
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    two_sum_acc(hi[a][b], lo[a][b], c[a][b]);
                    c[a][b] = 0.0f;
                }
        }
    }
    __device__ __forceinline__ double value(int a, int b) const {
        if constexpr (std::is_same<T, float>::value) return (double)hi[a][b] + (double)lo[a][b];
        else return c[a][b];
    }
    __device__ __forceinline__ void mma_chunk(const T (*As)[T_], const T (*Bs)[T_], int ty, int tx, int kc) {
#pragma unroll 8
        for (int kk = 0; kk < kc; kk++) {
            T ra[4], rb[4];
            lds4(&As[kk][ty * 4], ra);
            lds4(&Bs[kk][tx * 4], rb);
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) c[a][b] = fma(ra[a], rb[b], c[a][b]);
        }
    }
};

template <typename T>
__global__ void __launch_bounds__(256) h_simt_kernel(DevSystem s, const HWork *__restrict__ work,
                                                    const T *__restrict__ scratch, uint32_t terms) {
    constexpr int KC = Cfg<T>::KC;
    constexpr int VL = KC / 4;  // elements each thread loads per row segment
    __shared__ __align__(16) T As[KC][T_];
    __shared__ __align__(16) T Bs[KC][T_];
    __shared__ T dv[NAO_MAX_BATCH], dk[NAO_MAX_BATCH];  // weights of the potential and kinetic parts
    const HWork it = work[blockIdx.x];
    const int b = it.batch, m = s.sys.bmol[b];
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const int64_t ld = 4 * (int64_t)Ppad;
    const T *E = scratch + s.scr_off[b];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;

    for (int q = tid; q < Ppad; q += blockDim.x) {
        const double w = q < P ? s.pw[p0 + q] : 0.0;
        const double vv = q < P ? v_at(s, m, p0 + q) : 1.0;
        dv[q] = T((terms & NAO_TERM_POTENTIAL) ? w * vv : 0.0);
        const double kin = (terms & NAO_TERM_KINETIC) ? 1.0 : 0.0;
        dk[q] = T(0.5 * w * ((terms & NAO_TERM_TAU) && q < P ? kin + vt_at(s, m, p0 + q) : kin));
    }

    const int i0 = it.ti * T_, j0 = it.tj * T_;
    const int lrow = tid >> 2, lk = (tid & 3) * VL;
    const bool arow_ok = i0 + lrow < N, brow_ok = j0 + lrow < N;
    const T *Arow = E + (int64_t)(i0 + lrow) * ld + lk;
    const T *Brow = E + (int64_t)(j0 + lrow) * ld + lk;

    Block<T> acc;
    acc.zero();
    __syncthreads();
    const int K = 4 * Ppad;
    for (int k0 = 0; k0 < K; k0 += KC) {
        T av[VL], bv[VL];
#pragma unroll
        for (int u = 0; u < VL; u++) av[u] = bv[u] = T(0);
        if (arow_ok) load_vec(Arow + k0, av);
        if (brow_ok) load_vec(Brow + k0, bv);
#pragma unroll
        for (int u = 0; u < VL; u++) {
            // column k of E belongs to component k / Ppad (phi, d/dx, d/dy, d/dz) of point k % Ppad;
            // a chunk may straddle two components when Ppad is not a multiple of KC
            const int k = k0 + lk + u, comp = k / Ppad, q = k - comp * Ppad;
            As[lk + u][lrow] = av[u];
            Bs[lk + u][lrow] = bv[u] * (comp == 0 ? dv[q] : dk[q]);
        }
        __syncthreads();
        acc.mma_chunk(As, Bs, ty, tx, KC);
        acc.fold();
        __syncthreads();
    }

    const int32_t *rel = s.rel_idx + s.rel_off[b];
    const bool diag = it.ti == it.tj;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int i = i0 + ty * 4 + a;
        if (i >= N) continue;
        const int64_t gi = rel[i];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const int j = j0 + tx * 4 + c;
            if (j >= N || (diag && j < i)) continue;
            h_add(s, m, gi, rel[j], acc.value(a, c));
        }
    }
}

// Copy the upper triangle of each system's H onto its lower one, through 32 x 32 tiles; one
// CTA per task (system, column tile bx, row tile by) with by <= bx.
// In the deterministic mode the upper triangle comes from the fixed-point accumulators, converted
// once here (and written to both triangles).
__global__ void mirror_kernel(DevSystem s, const int4 *__restrict__ tasks) {
    __shared__ double tile[32][33];
    const int4 tk = tasks[blockIdx.x];
    const int m = tk.x, bx = tk.y, by = tk.z;
    double *H = s.sys.H[m];
    const unsigned long long *acc = s.sys.Hacc[m];
    const int64_t nb = s.sys.nbm[m];
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += blockDim.y) {
        const int64_t row = (int64_t)by * 32 + r, col = (int64_t)bx * 32 + tx;
        double h = 0.0;
        if (row < nb && col < nb) {
            if (acc) {
                if (row <= col) {
                    h = det_value(acc + 2 * (row * nb + col));
                    H[row * nb + col] = h;
                }
            } else {
                h = H[row * nb + col];
            }
        }
        tile[r][tx] = h;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += blockDim.y) {
        const int64_t row = (int64_t)bx * 32 + r, col = (int64_t)by * 32 + tx;  // destination, lower part
        if (row < nb && col < nb && row > col) H[row * nb + col] = tile[tx][r];
    }
}

// H = 0 for each task (system, first element, count); in the deterministic mode its fixed-point
// accumulators instead (H itself is then written whole by the mirror pass).
__global__ void __launch_bounds__(256) zero_h_kernel(DevSystem s, const int4 *__restrict__ tasks) {
    const int4 tk = tasks[blockIdx.x];
    unsigned long long *acc = s.sys.Hacc[tk.x];
    if (acc) {
        acc += 2 * ((int64_t)tk.y * 65536);
        for (int i = threadIdx.x; i < 2 * tk.z; i += blockDim.x) acc[i] = 0ULL;
        return;
    }
    double *H = s.sys.H[tk.x] + (int64_t)tk.y * 65536;
    for (int i = threadIdx.x; i < tk.z; i += blockDim.x) H[i] = 0.0;
}

// GRADN: the density gradient too (Sec. 2; grad n = 2 sum_ij grad phi_i P_ij phi_j): with
// T_qj = sum_i phi_qi P_ij over all of P (no tile-pair symmetry), n_q = sum_j T_qj phi_qj and
// grad n_q = 2 sum_j T_qj grad phi_qj; the scratch rows then hold [phi | d/dx | d/dy | d/dz].
template <typename T, bool GRADN>
__global__ void __launch_bounds__(256) density_simt_kernel(DevSystem s, const DWork *__restrict__ work, int32_t w0,
                                                          const T *__restrict__ scratch, double *__restrict__ ne_part) {
    constexpr int KC = Cfg<T>::KC;
    constexpr int RPT = (KC * T_) / 256;     // elements each thread loads per tile
    __shared__ __align__(16) T As[KC][T_];  // phi[i][q]
    __shared__ __align__(16) T Bs[KC][T_];  // c_IJ P[rel_i][rel_j]
    __shared__ double nacc[T_];
    __shared__ double gacc[GRADN ? 3 : 1][T_];
    __shared__ double red[8];
    const DWork it = work[w0 + blockIdx.x];
    const int b = it.batch, m = s.sys.bmol[b];
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    const int q0 = it.tp * T_;
    const T *E = scratch + s.scr_off[b];  // row stride Ppad (phi only) or 4 Ppad (GRADN)
    const int64_t ld = GRADN ? 4 * (int64_t)Ppad : (int64_t)Ppad;
    const int32_t *rel = s.rel_idx + s.rel_off[b];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int nt = (N + T_ - 1) / T_;
    if (tid < T_) {
        nacc[tid] = 0.0;
        if (GRADN) gacc[0][tid] = gacc[GRADN ? 1 : 0][tid] = gacc[GRADN ? 2 : 0][tid] = 0.0;
    }

    // loader mapping: row lk of the chunk, RPT consecutive columns starting at lc
    const int lk = tid / (T_ / RPT), lc = (tid % (T_ / RPT)) * RPT;
    for (int tj = 0; tj < nt; tj++) {
        Block<T> acc;
        acc.zero();
        for (int ti = 0; ti < (GRADN ? nt : tj + 1); ti++) {
            const double scale = (!GRADN && ti < tj) ? 2.0 : 1.0;
            for (int k0 = 0; k0 < T_; k0 += KC) {
                const int i = ti * T_ + k0 + lk;
                T fv[RPT];
#pragma unroll
                for (int u = 0; u < RPT; u++) fv[u] = T(0);
                if (i < N && q0 + lc < Ppad) load_vec(E + (int64_t)i * ld + q0 + lc, fv);
#pragma unroll
                for (int u = 0; u < RPT; u++) {
                    As[lk][lc + u] = fv[u];
                    const int j = tj * T_ + lc + u;
                    T pv = T(0);
                    if (i < N && j < N) {
                        int64_t gi = rel[i], gj = rel[j];
                        if (gi > gj) { const int64_t t = gi; gi = gj; gj = t; }
                        pv = T(scale * p_elem(s, m, gi, gj));
                    }
                    Bs[lk][lc + u] = pv;
                }
                __syncthreads();
                acc.mma_chunk(As, Bs, ty, tx, KC);
                acc.fold();
                __syncthreads();
            }
        }
        // n_q += sum_{j in J} T_qj phi_jq  (rows q = ty*4 + a of the tile, columns j = tx*4 + c)
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int q = q0 + ty * 4 + a;
            double part = 0.0, gp[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int j = tj * T_ + tx * 4 + c;
                const bool ok = j < N && q < Ppad;
                const double tv = acc.value(a, c);
                part += tv * (ok ? (double)E[(int64_t)j * ld + q] : 0.0);
                if (GRADN)
#pragma unroll
                    for (int d = 0; d < 3; d++) gp[d] += tv * (ok ? (double)E[(int64_t)j * ld + (d + 1) * Ppad + q] : 0.0);
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                part += __shfl_xor_sync(0xffffffffu, part, o);
                if (GRADN)
#pragma unroll
                    for (int d = 0; d < 3; d++) gp[d] += __shfl_xor_sync(0xffffffffu, gp[d], o);
            }
            if (tx == 0) {
                nacc[ty * 4 + a] += part;
                if (GRADN)
#pragma unroll
                    for (int d = 0; d < 3; d++) gacc[d][ty * 4 + a] += 2.0 * gp[d];
            }
        }
        __syncthreads();
    }
    __syncthreads();
    double wn = 0.0;
    if (tid < T_) {
        const int q = q0 + tid;
        if (q < P) {
            const double nv = nacc[tid];
            *n_at(s, m, p0 + q) = nv;
            if (GRADN)
#pragma unroll
                for (int d = 0; d < 3; d++) *gn_at(s, m, p0 + q, d) = gacc[d][tid];
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

// N_e of each system: one CTA per system sums its density work items' partial sums in a fixed
// assignment and tree order (deterministic).
__global__ void __launch_bounds__(1024) reduce_ne_kernel(DevSystem s, const double *__restrict__ part,
                                                        const int32_t *__restrict__ sys_dw0) {
    __shared__ double red[32];
    const int m = blockIdx.x;
    double *out = s.sys.ne[m];
    if (!out) return;
    double t = 0.0;
    for (int64_t i = sys_dw0[m] + threadIdx.x; i < sys_dw0[m + 1]; i += blockDim.x) t += part[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x < 32) {
        t = red[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) out[0] = t;
    }
}

// Pointer-table entries passed by value in the kernel's arguments.
constexpr int kPtrBatch = 480;
struct PtrBatch {
    void *p[kPtrBatch];
};
__global__ void set_pointers_kernel(double **__restrict__ dst, PtrBatch src, int32_t n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = static_cast<double *>(src.p[i]);
}

// n = 0 (and grad n = 0) at the points of each density work item: the tensor-core density
// writes only the points of batches that have basis functions.
__global__ void __launch_bounds__(64) zero_n_kernel(DevSystem s, const DWork *__restrict__ work, int grad) {
    const DWork it = work[blockIdx.x];
    const int p0 = s.batch_off[it.batch], P = s.batch_off[it.batch + 1] - p0;
    const int q = it.tp * NAO_TILE + threadIdx.x;
    if (q >= P) return;
    const int m = s.sys.bmol[it.batch];
    *n_at(s, m, p0 + q) = 0.0;
    if (grad)
        for (int d = 0; d < 3; d++) *gn_at(s, m, p0 + q, d) = 0.0;
}

}  // namespace

cudaError_t launch_h_simt(const DevSystem &s, nao_precision prec, const HWork *work, int32_t n_work,
                          const double *scratch, uint32_t terms, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    if (prec == NAO_FP32)
        h_simt_kernel<float><<<n_work, 256, 0, st>>>(s, work, reinterpret_cast<const float *>(scratch), terms);
    else
        h_simt_kernel<double><<<n_work, 256, 0, st>>>(s, work, scratch, terms);
    return cudaGetLastError();
}

cudaError_t launch_zero_h(const DevSystem &s, const int4 *tasks, int32_t n_tasks, cudaStream_t st) {
    if (n_tasks <= 0) return cudaSuccess;
    zero_h_kernel<<<n_tasks, 256, 0, st>>>(s, tasks);
    return cudaGetLastError();
}

cudaError_t launch_mirror(const DevSystem &s, const int4 *tasks, int32_t n_tasks, cudaStream_t st) {
    if (n_tasks <= 0) return cudaSuccess;
    mirror_kernel<<<n_tasks, dim3(32, 8), 0, st>>>(s, tasks);
    return cudaGetLastError();
}

cudaError_t launch_density_simt(const DevSystem &s, nao_precision prec, const DWork *work, int32_t w0, int32_t n_work,
                                const double *scratch, double *ne_part, bool grad, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    const float *sf = reinterpret_cast<const float *>(scratch);
    if (prec == NAO_FP32 && grad) density_simt_kernel<float, true><<<n_work, 256, 0, st>>>(s, work, w0, sf, ne_part);
    else if (prec == NAO_FP32) density_simt_kernel<float, false><<<n_work, 256, 0, st>>>(s, work, w0, sf, ne_part);
    else if (grad) density_simt_kernel<double, true><<<n_work, 256, 0, st>>>(s, work, w0, scratch, ne_part);
    else density_simt_kernel<double, false><<<n_work, 256, 0, st>>>(s, work, w0, scratch, ne_part);
    return cudaGetLastError();
}

cudaError_t launch_reduce_ne(const DevSystem &s, const double *part, const int32_t *sys_dw0, int32_t n_sys,
                             cudaStream_t st) {
    if (n_sys <= 0) return cudaSuccess;
    reduce_ne_kernel<<<n_sys, 1024, 0, st>>>(s, part, sys_dw0);
    return cudaGetLastError();
}

cudaError_t launch_set_pointers(double **dst, void *const *src, int32_t n, cudaStream_t st) {
    for (int32_t i0 = 0; i0 < n; i0 += kPtrBatch) {
        const int32_t c = n - i0 < kPtrBatch ? n - i0 : kPtrBatch;
        PtrBatch b;
        for (int32_t i = 0; i < c; i++) b.p[i] = src[i0 + i];
        set_pointers_kernel<<<1, 128, 0, st>>>(dst + i0, b, c);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_zero_n(const DevSystem &s, const DWork *work, int32_t n_work, bool grad, cudaStream_t st) {
    if (n_work <= 0) return cudaSuccess;
    zero_n_kernel<<<n_work, 64, 0, st>>>(s, work, grad ? 1 : 0);
    return cudaGetLastError();
}

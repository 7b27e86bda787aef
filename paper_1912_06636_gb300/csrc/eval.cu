// Evaluation phase (Sec. 3.4): basis functions phi_i and their gradients on each batch's
// points, for the functions of the batch's reduced basis nnz(B) (Sec. 3.3.2); and the
// batch-to-atom distances behind nnz(B).
//
// phi_i(r) = R_f(|d|) Y_lm(d/|d|), d = r - R_A, is computed as g(r) S_lm(d) with the real
// solid harmonic S_lm = r^l Y_lm (a polynomial in x, y, z) and g = R / r^l, so that
//   grad phi = g'(r) (d/r) S_lm + g grad S_lm,   g' = (R' - l R / r) / r^l.
// S_lm comes from the recurrences
//   Pi_m^m = (2m-1)!!,  Pi_{m+1}^m = (2m+1) z Pi_m^m,
//   (l-m) Pi_l^m = (2l-1) z Pi_{l-1}^m - (l+m-1) r^2 Pi_{l-2}^m,
//   A_m + i B_m = (x + i y)^m,
//   S_l0 = K_l0 Pi_l^0,  S_lm = sqrt2 K_lm Pi_l^m A_m,  S_l,-m = sqrt2 K_lm Pi_l^m B_m,
// carried together with their derivatives in z and in r^2, so that no division by sin(theta)
// occurs anywhere. R_f is the natural cubic spline in s = ln(r/r0)/Delta, evaluated as a
// per-segment polynomial in t = s - floor(s) (r < r0 uses r0; R = 0 for r >= rc).
#include <cmath>
#include <type_traits>

#include "nao_internal.h"

namespace {

// (2m-1)!!
__host__ __device__ constexpr double double_factorial_odd(int m) { return m <= 1 ? 1.0 : (2 * m - 1) * double_factorial_odd(m - 1); }

// ----------------------------------------------------------------------------------------
// nnz(B): min over each batch's points of |r - R_A|^2 per atom, every operation separately
// rounded (the host then applies r2 < rc*rc per radial function). One warp per atom.
// ----------------------------------------------------------------------------------------
__global__ void minr2_kernel(const double *__restrict__ atom_xyz, int n_atoms, const double *__restrict__ px,
                             const double *__restrict__ py, const double *__restrict__ pz,
                             const int32_t *__restrict__ boff, double *__restrict__ minr2) {
    const int b = blockIdx.x;
    const int p0 = boff[b], p1 = boff[b + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int a = warp; a < n_atoms; a += nwarp) {
        const double ax = atom_xyz[3 * a], ay = atom_xyz[3 * a + 1], az = atom_xyz[3 * a + 2];
        double m = __longlong_as_double(0x7ff0000000000000LL);  // +inf
        for (int p = p0 + lane; p < p1; p += 32) {
            const double dx = __dsub_rn(px[p], ax), dy = __dsub_rn(py[p], ay), dz = __dsub_rn(pz[p], az);
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            m = fmin(m, r2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) minr2[(size_t)b * n_atoms + a] = m;
    }
}

// ----------------------------------------------------------------------------------------
// solid harmonics of degree L with gradients (T = double or float)
// ----------------------------------------------------------------------------------------
template <int L, typename T>
__device__ __forceinline__ void solid_harmonics(T x, T y, T z, T q, const DevSystem &s, T (&S)[2 * L + 1],
                                                T (&Gx)[2 * L + 1], T (&Gy)[2 * L + 1], T (&Gz)[2 * L + 1]) {
    T A = T(1), B = T(0), Ap = T(0), Bp = T(0);
#pragma unroll
    for (int m = 0; m <= L; m++) {
        T p = T(double_factorial_odd(m)), pz = T(0), pq = T(0);
        if (L > m) {
            T p2 = p, p2z = T(0), p2q = T(0);
            T p1 = T(2 * m + 1) * z * p, p1z = T(2 * m + 1) * p, p1q = T(0);
#pragma unroll
            for (int l = m + 2; l <= L; l++) {
                const T c1 = T((double)(2 * l - 1) / (double)(l - m));
                const T c2 = T((double)(l + m - 1) / (double)(l - m));
                const T pn = c1 * z * p1 - c2 * q * p2;
                const T pnz = c1 * (p1 + z * p1z) - c2 * q * p2z;
                const T pnq = c1 * z * p1q - c2 * (p2 + q * p2q);
                p2 = p1; p2z = p1z; p2q = p1q;
                p1 = pn; p1z = pnz; p1q = pnq;
            }
            p = p1; pz = p1z; pq = p1q;
        }
        const T dPx = T(2) * x * pq, dPy = T(2) * y * pq, dPz = pz + T(2) * z * pq;
        const T kn = T(s.knorm[L][m]);
        if (m == 0) {
            S[L] = kn * p;
            Gx[L] = kn * dPx;
            Gy[L] = kn * dPy;
            Gz[L] = kn * dPz;
        } else {
            const T fm = T(m);
            S[L + m] = kn * p * A;
            Gx[L + m] = kn * (dPx * A + p * fm * Ap);
            Gy[L + m] = kn * (dPy * A - p * fm * Bp);
            Gz[L + m] = kn * dPz * A;
            S[L - m] = kn * p * B;
            Gx[L - m] = kn * (dPx * B + p * fm * Bp);
            Gy[L - m] = kn * (dPy * B + p * fm * Ap);
            Gz[L - m] = kn * dPz * B;
        }
        Ap = A;
        Bp = B;
        A = x * Ap - y * Bp;
        B = x * Bp + y * Ap;
    }
}

// R and dR/dr in FP64: s = ln(max(r, r0)/r0)/Delta, segment k = floor(s), t = s - k.
__device__ __forceinline__ void radial_f64(const DevSystem &s, int fn, double r, double &R, double &dR) {
    const double rr = fmax(r, s.r0);
    const double sc = log(rr / s.r0) * s.inv_delta;
    int k = (int)floor(sc);
    k = k < 0 ? 0 : (k > s.n_rgrid - 2 ? s.n_rgrid - 2 : k);
    const double t = sc - (double)k;
    const double2 *c = reinterpret_cast<const double2 *>(s.coef + ((size_t)fn * (s.n_rgrid - 1) + k) * 4);
    const double2 c01 = __ldg(c), c23 = __ldg(c + 1);
    R = fma(fma(fma(c23.y, t, c23.x), t, c01.y), t, c01.x);
    dR = fma(fma(3.0 * c23.y, t, 2.0 * c23.x), t, c01.y) * s.inv_delta / rr;
}

// R and dR/dr in FP32. The segment comes from an FP32 logarithm; t is then refined as
// ln(r / r_k)/Delta = log1p(r * (1/r_k) - 1)/Delta with r and 1/r_k in FP64 (one FMA), so
// that t is accurate to ~1e-7 although r itself only has FP32's relative precision in the
// rest of the evaluation (for steep functions ln R changes ~2 alpha r^2 times faster than r).
__device__ __forceinline__ void radial_f32(const DevSystem &s, int fn, double r64, float &R, float &dR) {
    const double rr64 = fmax(r64, s.r0);
    const float rr = (float)rr64;
    const float sa = __logf(rr * (float)(1.0 / s.r0)) * (float)s.inv_delta;
    int k = (int)floorf(sa);
    k = k < 0 ? 0 : (k > s.n_rgrid - 2 ? s.n_rgrid - 2 : k);
    const double x = fma(rr64, __ldg(s.inv_rk + k), -1.0);
    const float t = log1pf((float)x) * (float)s.inv_delta;
    const float4 c = __ldg(reinterpret_cast<const float4 *>(s.coef_f32 + ((size_t)fn * (s.n_rgrid - 1) + k) * 4));
    R = fmaf(fmaf(fmaf(c.w, t, c.z), t, c.y), t, c.x);
    dR = fmaf(fmaf(3.0f * c.w, t, 2.0f * c.z), t, c.y) * (float)s.inv_delta / rr;
}

// phi and grad phi of the 2L+1 functions of one radial function at one point.
template <int L, typename T>
__device__ __forceinline__ void basis_values(const DevSystem &s, int fn, T dx, T dy, T dz, T r2, T r, T R, T dR,
                                             T (&phi)[2 * L + 1], T (&gx)[2 * L + 1], T (&gy)[2 * L + 1],
                                             T (&gz)[2 * L + 1]) {
    T S[2 * L + 1], Gx[2 * L + 1], Gy[2 * L + 1], Gz[2 * L + 1];
    solid_harmonics<L, T>(dx, dy, dz, r2, s, S, Gx, Gy, Gz);
    const T u = T(1) / r;
    T ul = T(1);
#pragma unroll
    for (int i = 0; i < L; i++) ul *= u;
    const T g = R * ul;
    const T gpu = (dR - T(L) * R * u) * ul * u;  // g'(r) / r
#pragma unroll
    for (int m = 0; m < 2 * L + 1; m++) {
        phi[m] = g * S[m];
        gx[m] = gpu * dx * S[m] + g * Gx[m];
        gy[m] = gpu * dy * S[m] + g * Gy[m];
        gz[m] = gpu * dz * S[m] + g * Gz[m];
    }
}

// Output addressing of one evaluation launch.
template <typename OutT>
struct EvalOut {
    OutT *phi;    // phi of reduced-basis position j, point q at phi[j*phi_rs + q]
    OutT *grad;   // component c at grad[c*grad_cs + j*grad_rs + q] (nullptr: none)
    int64_t phi_rs, grad_cs, grad_rs;
    int32_t qmax; // points written per row (q >= P_b is written as 0)
};

// Distance below which the FP32 path evaluates in FP64 (bohr).
constexpr double kNearNucleus = 0.1;

template <int L, bool GRAD, typename T, typename OutT>
__device__ __forceinline__ void eval_one(const DevSystem &s, const RfnEntry &e, double dx, double dy, double dz,
                                         double r2, bool inside, const EvalOut<OutT> &o, int q) {
    OutT phi[2 * L + 1], gx[2 * L + 1], gy[2 * L + 1], gz[2 * L + 1];
#pragma unroll
    for (int m = 0; m < 2 * L + 1; m++) phi[m] = gx[m] = gy[m] = gz[m] = OutT(0);
    if (inside) {
        const double r = __dsqrt_rn(r2);
        if (std::is_same<T, double>::value || r < kNearNucleus) {
            double R, dR, f[2 * L + 1], a[2 * L + 1], b[2 * L + 1], c[2 * L + 1];
            radial_f64(s, e.fn, r, R, dR);
            basis_values<L, double>(s, e.fn, dx, dy, dz, r2, r, R, dR, f, a, b, c);
#pragma unroll
            for (int m = 0; m < 2 * L + 1; m++) {
                phi[m] = OutT(f[m]); gx[m] = OutT(a[m]); gy[m] = OutT(b[m]); gz[m] = OutT(c[m]);
            }
        } else {
            float R, dR, f[2 * L + 1], a[2 * L + 1], b[2 * L + 1], c[2 * L + 1];
            radial_f32(s, e.fn, r, R, dR);
            const float fx = (float)dx, fy = (float)dy, fz = (float)dz;
            basis_values<L, float>(s, e.fn, fx, fy, fz, (float)r2, (float)r, R, dR, f, a, b, c);
#pragma unroll
            for (int m = 0; m < 2 * L + 1; m++) {
                phi[m] = OutT(f[m]); gx[m] = OutT(a[m]); gy[m] = OutT(b[m]); gz[m] = OutT(c[m]);
            }
        }
    }
#pragma unroll
    for (int m = 0; m < 2 * L + 1; m++) {
        const int64_t j = e.pos + m;
        o.phi[j * o.phi_rs + q] = phi[m];
        if (GRAD) {
            o.grad[j * o.grad_rs + q] = gx[m];
            o.grad[o.grad_cs + j * o.grad_rs + q] = gy[m];
            o.grad[2 * o.grad_cs + j * o.grad_rs + q] = gz[m];
        }
    }
}

template <bool GRAD, typename T, typename OutT>
__device__ __forceinline__ void eval_batch(const DevSystem &s, int b, const EvalOut<OutT> &o) {
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int r0 = s.rfn_off[b], nr = s.rfn_off[b + 1] - r0;
    const int qmax = o.qmax;
    const int total = nr * qmax;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int rl = idx / qmax, q = idx - rl * qmax;
        const RfnEntry e = s.rfn[r0 + rl];
        double dx = 0.0, dy = 0.0, dz = 0.0, r2 = 0.0;
        bool inside = false;
        if (q < P) {
            const int p = p0 + q;
            dx = __dsub_rn(s.px[p], s.atom_xyz[3 * e.atom]);
            dy = __dsub_rn(s.py[p], s.atom_xyz[3 * e.atom + 1]);
            dz = __dsub_rn(s.pz[p], s.atom_xyz[3 * e.atom + 2]);
            r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            inside = __dsqrt_rn(r2) < s.fn_rc[e.fn];
        }
        switch (e.l) {
            case 0: eval_one<0, GRAD, T>(s, e, dx, dy, dz, r2, inside, o, q); break;
            case 1: eval_one<1, GRAD, T>(s, e, dx, dy, dz, r2, inside, o, q); break;
            case 2: eval_one<2, GRAD, T>(s, e, dx, dy, dz, r2, inside, o, q); break;
            case 3: eval_one<3, GRAD, T>(s, e, dx, dy, dz, r2, inside, o, q); break;
            case 4: eval_one<4, GRAD, T>(s, e, dx, dy, dz, r2, inside, o, q); break;
            case 5: eval_one<5, GRAD, T>(s, e, dx, dy, dz, r2, inside, o, q); break;
            default: eval_one<6, GRAD, T>(s, e, dx, dy, dz, r2, inside, o, q); break;
        }
    }
}

// One CTA per batch; the batch's block of scratch holds, per reduced-basis row j,
// [phi | d/dx | d/dy | d/dz] over Ppad points each (GRAD) or phi alone, in type T.
template <bool GRAD, typename T>
__global__ void __launch_bounds__(256) eval_chunk_kernel(DevSystem s, int32_t b0, T *scratch) {
    const int b = b0 + blockIdx.x;
    const int P = s.batch_off[b + 1] - s.batch_off[b];
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    EvalOut<T> o;
    o.phi = scratch + s.scr_off[b];
    o.qmax = Ppad;
    if (GRAD) {
        o.phi_rs = 4 * (int64_t)Ppad;
        o.grad = o.phi + Ppad;
        o.grad_cs = Ppad;
        o.grad_rs = 4 * (int64_t)Ppad;
    } else {
        o.phi_rs = Ppad;
        o.grad = nullptr;
        o.grad_cs = o.grad_rs = 0;
    }
    eval_batch<GRAD, T>(s, b, o);
}

template <bool GRAD, typename T>
__global__ void __launch_bounds__(256) eval_export_kernel(DevSystem s, int32_t b, double *phi, double *grad) {
    const int P = s.batch_off[b + 1] - s.batch_off[b];
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    EvalOut<double> o;
    o.phi = phi;
    o.phi_rs = P;
    o.grad = grad;
    o.grad_cs = (int64_t)N * P;
    o.grad_rs = P;
    o.qmax = P;
    eval_batch<GRAD, T>(s, b, o);
}

}  // namespace

cudaError_t launch_relevance_minr2(const double *atom_xyz, int32_t n_atoms, const double *px, const double *py,
                                   const double *pz, const int32_t *batch_off, int64_t n_batches, double *minr2,
                                   cudaStream_t st) {
    if (n_batches <= 0) return cudaSuccess;
    minr2_kernel<<<(unsigned)n_batches, 256, 0, st>>>(atom_xyz, n_atoms, px, py, pz, batch_off, minr2);
    return cudaGetLastError();
}

cudaError_t launch_eval(const DevSystem &s, int32_t b0, int32_t b1, nao_precision prec, bool grad, double *scratch,
                        cudaStream_t st) {
    if (b1 <= b0) return cudaSuccess;
    if (prec == NAO_FP32) {
        float *f = reinterpret_cast<float *>(scratch);
        if (grad) eval_chunk_kernel<true, float><<<b1 - b0, 256, 0, st>>>(s, b0, f);
        else eval_chunk_kernel<false, float><<<b1 - b0, 256, 0, st>>>(s, b0, f);
    } else {
        if (grad) eval_chunk_kernel<true, double><<<b1 - b0, 256, 0, st>>>(s, b0, scratch);
        else eval_chunk_kernel<false, double><<<b1 - b0, 256, 0, st>>>(s, b0, scratch);
    }
    return cudaGetLastError();
}

cudaError_t launch_eval_one(const DevSystem &s, int32_t b, nao_precision prec, double *phi, double *grad,
                            cudaStream_t st) {
    if (prec == NAO_FP32) {
        if (grad) eval_export_kernel<true, float><<<1, 256, 0, st>>>(s, b, phi, grad);
        else eval_export_kernel<false, float><<<1, 256, 0, st>>>(s, b, phi, nullptr);
    } else {
        if (grad) eval_export_kernel<true, double><<<1, 256, 0, st>>>(s, b, phi, grad);
        else eval_export_kernel<false, double><<<1, 256, 0, st>>>(s, b, phi, nullptr);
    }
    return cudaGetLastError();
}

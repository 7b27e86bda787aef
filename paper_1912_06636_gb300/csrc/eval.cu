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
// solid harmonics of degree L with gradients
// ----------------------------------------------------------------------------------------
template <int L>
__device__ __forceinline__ void solid_harmonics(double x, double y, double z, double q, const DevSystem &s,
                                                double (&S)[2 * L + 1], double (&Gx)[2 * L + 1],
                                                double (&Gy)[2 * L + 1], double (&Gz)[2 * L + 1]) {
    double A = 1.0, B = 0.0, Ap = 0.0, Bp = 0.0;
#pragma unroll
    for (int m = 0; m <= L; m++) {
        double p = double_factorial_odd(m), pz = 0.0, pq = 0.0;
        if (L > m) {
            double p2 = p, p2z = 0.0, p2q = 0.0;
            double p1 = (2 * m + 1) * z * p, p1z = (2 * m + 1) * p, p1q = 0.0;
#pragma unroll
            for (int l = m + 2; l <= L; l++) {
                const double c1 = (double)(2 * l - 1) / (double)(l - m);
                const double c2 = (double)(l + m - 1) / (double)(l - m);
                const double pn = c1 * z * p1 - c2 * q * p2;
                const double pnz = c1 * (p1 + z * p1z) - c2 * q * p2z;
                const double pnq = c1 * z * p1q - c2 * (p2 + q * p2q);
                p2 = p1; p2z = p1z; p2q = p1q;
                p1 = pn; p1z = pnz; p1q = pnq;
            }
            p = p1; pz = p1z; pq = p1q;
        }
        const double dPx = 2.0 * x * pq, dPy = 2.0 * y * pq, dPz = pz + 2.0 * z * pq;
        const double kn = s.knorm[L][m];
        if (m == 0) {
            S[L] = kn * p;
            Gx[L] = kn * dPx;
            Gy[L] = kn * dPy;
            Gz[L] = kn * dPz;
        } else {
            const double fm = (double)m;
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

// Output addressing of one evaluation launch.
struct EvalOut {
    double *phi;       // phi of reduced-basis position j, point q at phi[j*phi_rs + q]
    double *grad;      // component c at grad[c*grad_cs + j*grad_rs + q] (nullptr: none)
    int64_t phi_rs, grad_cs, grad_rs;
    int32_t qmax;      // points written per row (q >= P_b is written as 0)
};

template <int L, bool GRAD>
__device__ __forceinline__ void eval_one(const DevSystem &s, const RfnEntry &e, double dx, double dy, double dz,
                                         double r2, bool inside, const EvalOut &o, int q) {
    double S[2 * L + 1], Gx[2 * L + 1], Gy[2 * L + 1], Gz[2 * L + 1];
    double g = 0.0, gp = 0.0, u = 0.0;
    if (inside) {
        const double r = __dsqrt_rn(r2);
        const double rr = fmax(r, s.r0);
        const double sc = log(rr / s.r0) * s.inv_delta;
        int k = (int)floor(sc);
        k = k < 0 ? 0 : (k > s.n_rgrid - 2 ? s.n_rgrid - 2 : k);
        const double t = sc - (double)k;
        const double2 *c = reinterpret_cast<const double2 *>(s.coef + ((size_t)e.fn * (s.n_rgrid - 1) + k) * 4);
        const double2 c01 = __ldg(c), c23 = __ldg(c + 1);
        const double R = fma(fma(fma(c23.y, t, c23.x), t, c01.y), t, c01.x);
        const double dR = fma(fma(3.0 * c23.y, t, 2.0 * c23.x), t, c01.y) * s.inv_delta / rr;
        u = 1.0 / r;
        double ul = 1.0;
#pragma unroll
        for (int i = 0; i < L; i++) ul *= u;
        g = R * ul;
        gp = (dR - (double)L * R * u) * ul;
        solid_harmonics<L>(dx, dy, dz, r2, s, S, Gx, Gy, Gz);
    } else {
#pragma unroll
        for (int m = 0; m < 2 * L + 1; m++) S[m] = Gx[m] = Gy[m] = Gz[m] = 0.0;
    }
    const double gpu = gp * u;
#pragma unroll
    for (int m = 0; m < 2 * L + 1; m++) {
        const int64_t j = e.pos + m;
        o.phi[j * o.phi_rs + q] = g * S[m];
        if (GRAD) {
            o.grad[j * o.grad_rs + q] = fma(gpu * dx, S[m], g * Gx[m]);
            o.grad[o.grad_cs + j * o.grad_rs + q] = fma(gpu * dy, S[m], g * Gy[m]);
            o.grad[2 * o.grad_cs + j * o.grad_rs + q] = fma(gpu * dz, S[m], g * Gz[m]);
        }
    }
}

template <bool GRAD>
__device__ __forceinline__ void eval_batch(const DevSystem &s, int b, const EvalOut &o) {
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
            case 0: eval_one<0, GRAD>(s, e, dx, dy, dz, r2, inside, o, q); break;
            case 1: eval_one<1, GRAD>(s, e, dx, dy, dz, r2, inside, o, q); break;
            case 2: eval_one<2, GRAD>(s, e, dx, dy, dz, r2, inside, o, q); break;
            case 3: eval_one<3, GRAD>(s, e, dx, dy, dz, r2, inside, o, q); break;
            case 4: eval_one<4, GRAD>(s, e, dx, dy, dz, r2, inside, o, q); break;
            case 5: eval_one<5, GRAD>(s, e, dx, dy, dz, r2, inside, o, q); break;
            default: eval_one<6, GRAD>(s, e, dx, dy, dz, r2, inside, o, q); break;
        }
    }
}

// One CTA per batch; the batch's block of scratch holds, per reduced-basis row j,
// [phi | d/dx | d/dy | d/dz] over Ppad points each (GRAD) or phi alone.
template <bool GRAD>
__global__ void __launch_bounds__(256) eval_chunk_kernel(DevSystem s, int32_t b0, double *scratch) {
    const int b = b0 + blockIdx.x;
    const int P = s.batch_off[b + 1] - s.batch_off[b];
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    EvalOut o;
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
    eval_batch<GRAD>(s, b, o);
}

template <bool GRAD>
__global__ void __launch_bounds__(256) eval_export_kernel(DevSystem s, int32_t b, double *phi, double *grad) {
    const int P = s.batch_off[b + 1] - s.batch_off[b];
    const int N = s.rel_off[b + 1] - s.rel_off[b];
    EvalOut o;
    o.phi = phi;
    o.phi_rs = P;
    o.grad = grad;
    o.grad_cs = (int64_t)N * P;
    o.grad_rs = P;
    o.qmax = P;
    eval_batch<GRAD>(s, b, o);
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
    (void)prec;
    if (b1 <= b0) return cudaSuccess;
    if (grad) eval_chunk_kernel<true><<<b1 - b0, 256, 0, st>>>(s, b0, scratch);
    else eval_chunk_kernel<false><<<b1 - b0, 256, 0, st>>>(s, b0, scratch);
    return cudaGetLastError();
}

cudaError_t launch_eval_one(const DevSystem &s, int32_t b, nao_precision prec, double *phi, double *grad,
                            cudaStream_t st) {
    (void)prec;
    if (grad) eval_export_kernel<true><<<1, 256, 0, st>>>(s, b, phi, grad);
    else eval_export_kernel<false><<<1, 256, 0, st>>>(s, b, phi, nullptr);
    return cudaGetLastError();
}

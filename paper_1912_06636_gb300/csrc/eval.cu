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

#include "ff.h"
#include "nao_internal.h"
#include "split_bits.h"

namespace {

// log(1 + x) for the radial coordinate, x = r / r_k - 1, normally in [0, b), b = exp(Delta) - 1
// of the logarithmic grid. For |x| <= b <= 0.031 (grids with Delta <= 0.03) the Taylor series
// x - x^2/2 + x^3/3 - ... to x^12/12 (the first omitted term is below 2^-53 |x|), evaluated by
// Horner's rule; otherwise (coarser grids, r beyond the last knot) log1p.
__device__ __forceinline__ double log1p_small(double x, double b) {
    if (b > 0.031 || fabs(x) > b) return log1p(x);
    double p = -1.0 / 12.0;
    p = fma(p, x, 1.0 / 11.0);
    p = fma(p, x, -1.0 / 10.0);
    p = fma(p, x, 1.0 / 9.0);
    p = fma(p, x, -1.0 / 8.0);
    p = fma(p, x, 1.0 / 7.0);
    p = fma(p, x, -1.0 / 6.0);
    p = fma(p, x, 1.0 / 5.0);
    p = fma(p, x, -1.0 / 4.0);
    p = fma(p, x, 1.0 / 3.0);
    p = fma(p, x, -0.5);
    p = fma(p, x, 1.0);
    return p * x;
}

// (2m-1)!!
__host__ __device__ constexpr double double_factorial_odd(int m) { return m <= 1 ? 1.0 : (2 * m - 1) * double_factorial_odd(m - 1); }

// ----------------------------------------------------------------------------------------
// nnz(B): min over each batch's points of |r - R_A|^2 per atom, every operation separately
// rounded (the host then applies r2 < rc*rc per radial function). One warp per atom.
// ----------------------------------------------------------------------------------------
__global__ void minr2_kernel(const double *__restrict__ atom_xyz, const int32_t *__restrict__ bmol,
                             const int32_t *__restrict__ aoff, int max_atoms, const double *__restrict__ px,
                             const double *__restrict__ py, const double *__restrict__ pz,
                             const int32_t *__restrict__ boff, double *__restrict__ minr2) {
    const int b = blockIdx.x, m = bmol[b];
    const int p0 = boff[b], p1 = boff[b + 1];
    const int a0 = aoff[m], na = aoff[m + 1] - a0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int a = warp; a < na; a += nwarp) {
        const double ax = atom_xyz[3 * (a0 + a)], ay = atom_xyz[3 * (a0 + a) + 1], az = atom_xyz[3 * (a0 + a) + 2];
        double mn = __longlong_as_double(0x7ff0000000000000LL);  // +inf
        for (int p = p0 + lane; p < p1; p += 32) {
            const double dx = __dsub_rn(px[p], ax), dy = __dsub_rn(py[p], ay), dz = __dsub_rn(pz[p], az);
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            mn = fmin(mn, r2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        if (lane == 0) minr2[(size_t)b * max_atoms + a] = mn;
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

// Split path (EXPO = 1): per point, the largest biased exponent of phi over the basis, reduced
// while the values are produced (the density slicing's point exponents) into red[q], shared
// memory of the batch's CTA.
struct ExpoIn {
    int *red;
};

// Distance below which the FP32 path evaluates in FP64 (bohr).
constexpr double kNearNucleus = 0.1;

template <typename OutT>
__device__ __forceinline__ void store_rows(const EvalOut<OutT> &o, int pos, int nm, int q, const OutT *phi,
                                           const OutT *gx, const OutT *gy, const OutT *gz, bool grad) {
    for (int m = 0; m < nm; m++) {
        const int64_t j = pos + m;
        o.phi[j * o.phi_rs + q] = phi[m];
        if (grad) {
            o.grad[j * o.grad_rs + q] = gx[m];
            o.grad[o.grad_cs + j * o.grad_rs + q] = gy[m];
            o.grad[2 * o.grad_cs + j * o.grad_rs + q] = gz[m];
        }
    }
}

// All relevant radial functions of one atom at one point, in arithmetic T. Distance, square
// root, logarithm, reciprocals and the solid-harmonic recurrence are shared by the atom's
// radial functions, which are visited in increasing l.
template <int LMAX, typename T, bool GRAD, typename OutT, int EXPO>
__device__ __noinline__ void eval_group(const DevSystem &s, const AtomGroup &ag, double dx, double dy, double dz,
                                           double r2, double r, double ur, const EvalOut<OutT> &o, int q,
                                           ExpoIn xi) {
    // radial coordinate: segment k and t in [0, 1)
    const double rr = fmax(r, s.r0);
    int k;
    T t;
    double xk = 0.0;  // FP32 path: r / r_k - 1, for the FP64 re-evaluation of ill-conditioned segments
    if constexpr (std::is_same<T, double>::value) {
        // segment k from an FP32 logarithm, moved by one where it disagrees with the FP64 knots
        // (r_k <= r < r_{k+1} as rr / r_k - 1 in [0, exp(Delta) - 1)), then
        // t = ln(r / r_k) / Delta = log1p(rr / r_k - 1) / Delta
        const float sa = __logf((float)rr * (float)__ldg(s.inv_rk)) * (float)s.inv_delta;
        k = (int)floorf(sa);
        k = k < 0 ? 0 : (k > s.n_rgrid - 2 ? s.n_rgrid - 2 : k);
        double xr = fma(rr, __ldg(s.inv_rk + k), -1.0);
        if (xr < 0.0 && k > 0) {
            k--;
            xr = fma(rr, __ldg(s.inv_rk + k), -1.0);
        } else if (xr >= s.step_m1 && k < s.n_rgrid - 2) {
            k++;
            xr = fma(rr, __ldg(s.inv_rk + k), -1.0);
        }
        t = log1p_small(xr, s.step_m1) * s.inv_delta;
    } else {
        // FP32 segment, refined as ln(r / r_k)/Delta = log1p(r * (1/r_k) - 1)/Delta with one FP64
        // FMA: t keeps ~1e-7 although a plain FP32 ln(r/r0) carries ~1e-6.
        const float sa = __logf((float)rr * (float)(1.0 / s.r0)) * (float)s.inv_delta;
        k = (int)floorf(sa);
        k = k < 0 ? 0 : (k > s.n_rgrid - 2 ? s.n_rgrid - 2 : k);
        xk = fma(rr, __ldg(s.inv_rk + k), -1.0);
        t = log1pf((float)xk) * (float)s.inv_delta;
    }
    const T dr_scale = T(s.inv_delta * (r < s.r0 ? __ldg(s.inv_rk) : ur));  // dR/dr = dR/ds * inv_delta / rr
    const T u = T(ur);
    const T x = T(dx), y = T(dy), z = T(dz);
    // The solid harmonics and their gradients are computed in FP64 on both paths (type H): the
    // recurrences cancel near the nodes of cos(m phi), sin(m phi) and P_l^m(cos theta), where
    // FP32 (with FP32-rounded x, y, z) loses several ulps; the FP32 path rounds the results once.
    using H = double;
    const H xh = dx, yh = dy, zh = dz, qq = r2;
    const H x2 = xh + xh, y2 = yh + yh, z2 = zh + zh;
    // A_m + i B_m = (x + i y)^m
    // (A_0, B_0) = (1, 0) and (A_1, B_1) = (x, y) exactly. Terms that vanish for every point
    // (a derivative of a constant or of a polynomial without that variable, a factor B_0) are
    // left out rather than multiplied by zero, which IEEE arithmetic would not let the compiler
    // drop: the flags below are compile-time constants once the loops over l and m unroll.
    H A[LMAX + 1], B[LMAX + 1];
    A[0] = H(1);
    B[0] = H(0);
#pragma unroll
    for (int m = 1; m <= LMAX; m++) {
        if (m == 1) {
            A[1] = xh;
            B[1] = yh;
        } else {
            A[m] = xh * A[m - 1] - yh * B[m - 1];
            B[m] = xh * B[m - 1] + yh * A[m - 1];
        }
    }
    // Pi_{l-1}^m (c) and Pi_{l-2}^m (p) with their z and r^2 derivatives. Pi_l^m is a
    // polynomial in z of degree l - m and in r^2 of degree floor((l - m) / 2): its z-derivative
    // vanishes for l = m, its r^2-derivative for l - m < 2.
    H Pc[LMAX + 1], Pcz[LMAX + 1], Pcq[LMAX + 1], Pp[LMAX + 1], Ppz[LMAX + 1], Ppq[LMAX + 1];
#pragma unroll
    for (int m = 0; m <= LMAX; m++) Pc[m] = Pcz[m] = Pcq[m] = Pp[m] = Ppz[m] = Ppq[m] = H(0);
    int ri = ag.r0;
    const int re = ag.r0 + ag.nr;
    int pt_eb = 0;  // EXPO 1: largest biased exponent of phi at this point
    T ul = T(1);  // u^l
#pragma unroll
    for (int l = 0; l <= LMAX; l++) {
        H S[2 * LMAX + 1], Gx[2 * LMAX + 1], Gy[2 * LMAX + 1], Gz[2 * LMAX + 1];
        bool zx[2 * LMAX + 1], zy[2 * LMAX + 1], zz[2 * LMAX + 1];  // gradient component is 0
#pragma unroll
        for (int m = 0; m <= l; m++) {
            H p, pz = H(0), pq = H(0);
            const bool zpz = (m == l), zpq = (l - m < 2);
            if (m == l) {
                p = H(double_factorial_odd(m));
            } else if (m == l - 1) {
                p = H(2 * m + 1) * zh * Pc[m];
                pz = H(2 * m + 1) * Pc[m];
            } else {
                const H c1 = H((double)(2 * l - 1) / (double)(l - m));
                const H c2 = H((double)(l + m - 1) / (double)(l - m));
                p = c1 * zh * Pc[m] - c2 * qq * Pp[m];
                pz = c1 * (Pc[m] + zh * Pcz[m]);
                if (l - 2 != m) pz = pz - c2 * qq * Ppz[m];          // Pi_{l-2}^m depends on z
                const H pq_p = (l - 2 - m >= 2) ? Pp[m] + qq * Ppq[m] : Pp[m];
                pq = (l - 1 - m >= 2) ? c1 * zh * Pcq[m] - c2 * pq_p : -(c2 * pq_p);
            }
            Pp[m] = Pc[m]; Ppz[m] = Pcz[m]; Ppq[m] = Pcq[m];
            Pc[m] = p; Pcz[m] = pz; Pcq[m] = pq;
            // K_lm folded into p and its derivatives once: kp = K p, kd = K grad(Pi)
            const H kn = H(s.knorm[l][m]);
            const H kp = kn * p;
            const H kpq = zpq ? H(0) : kn * pq;
            const H kdx = zpq ? H(0) : x2 * kpq, kdy = zpq ? H(0) : y2 * kpq;
            const H kdz = zpz ? (zpq ? H(0) : z2 * kpq) : (zpq ? kn * pz : fma(z2, kpq, kn * pz));
            const bool zdz = zpz && zpq;
            if (m == 0) {
                S[l] = kp;
                Gx[l] = kdx;
                Gy[l] = kdy;
                Gz[l] = kdz;
                zx[l] = zy[l] = zpq;
                zz[l] = zdz;
            } else {
                const H kpf = kp * H(m);
                S[l + m] = kp * A[m];
                Gx[l + m] = zpq ? kpf * A[m - 1] : fma(kdx, A[m], kpf * A[m - 1]);
                Gy[l + m] = m == 1 ? (zpq ? H(0) : kdy * A[m]) : (zpq ? -(kpf * B[m - 1]) : fma(kdy, A[m], -(kpf * B[m - 1])));
                Gz[l + m] = zdz ? H(0) : kdz * A[m];
                S[l - m] = kp * B[m];
                Gx[l - m] = m == 1 ? (zpq ? H(0) : kdx * B[m]) : (zpq ? kpf * B[m - 1] : fma(kdx, B[m], kpf * B[m - 1]));
                Gy[l - m] = zpq ? kpf * A[m - 1] : fma(kdy, B[m], kpf * A[m - 1]);
                Gz[l - m] = zdz ? H(0) : kdz * B[m];
                zx[l + m] = false;
                zy[l + m] = (m == 1 && zpq);
                zz[l + m] = zz[l - m] = zdz;
                zx[l - m] = (m == 1 && zpq);
                zy[l - m] = false;
            }
        }
        const T ulu = ul * u;                      // u^(l+1)
        const T a_dr = dr_scale * ulu;              // dR/ds -> g'(r)/r
        const T a_r = T(l) * u * ulu;               // R -> the l R / r part of g'(r)/r
        // the atom's radial functions of this l
        for (; ri < re; ri++) {
            const RfnEntry e = s.rfn[ri];
            if (e.l != l) break;
            OutT fo[2 * LMAX + 1], xo[2 * LMAX + 1], yo[2 * LMAX + 1], zo[2 * LMAX + 1];
            if (r < s.fn_rc[e.fn]) {
                T R, dRds;
                if constexpr (std::is_same<T, double>::value) {
                    const double2 *c = reinterpret_cast<const double2 *>(s.coef + ((size_t)e.fn * (s.n_rgrid - 1) + k) * 4);
                    const double2 c01 = __ldg(c), c23 = __ldg(c + 1);
                    // R = c0 + t (c1 + t a), dR/dt = c1 + t (2 a + c3 t), a = c2 + c3 t
                    const double a = fma(c23.y, t, c23.x);
                    R = fma(fma(a, t, c01.y), t, c01.x);
                    dRds = fma(fma(c23.y, t, a + a), t, c01.y);
                } else {
                    const size_t seg = (size_t)e.fn * (s.n_rgrid - 1) + k;
                    if (__ldg(s.seg64 + seg)) {
                        // ill-conditioned segment: FP64 coefficients and FP64 t
                        const double t64 = log1p(xk) * s.inv_delta;
                        const double2 *c = reinterpret_cast<const double2 *>(s.coef + seg * 4);
                        const double2 c01 = __ldg(c), c23 = __ldg(c + 1);
                        R = (float)fma(fma(fma(c23.y, t64, c23.x), t64, c01.y), t64, c01.x);
                        dRds = (float)fma(fma(3.0 * c23.y, t64, 2.0 * c23.x), t64, c01.y);
                    } else {
                        const float4 c = __ldg(reinterpret_cast<const float4 *>(s.coef_f32 + seg * 4));
                        R = fmaf(fmaf(fmaf(c.w, t, c.z), t, c.y), t, c.x);
                        dRds = fmaf(fmaf(3.0f * c.w, t, 2.0f * c.z), t, c.y);
                    }
                }
                const T g = R * ul;
                // g'(r) / r = (dR/dr - l R / r) u^l / r
                const T gpu = l == 0 ? dRds * a_dr : fma(dRds, a_dr, -(R * a_r));
                const T gx = gpu * x, gy = gpu * y, gz = gpu * z;
#pragma unroll
                for (int m = 0; m < 2 * l + 1; m++) {
                    const T Sm = T(S[m]);
                    fo[m] = OutT(g * Sm);
                    xo[m] = OutT(zx[m] ? gx * Sm : gx * Sm + g * T(Gx[m]));
                    yo[m] = OutT(zy[m] ? gy * Sm : gy * Sm + g * T(Gy[m]));
                    zo[m] = OutT(zz[m] ? gz * Sm : gz * Sm + g * T(Gz[m]));
                }
            } else {
#pragma unroll
                for (int m = 0; m < 2 * l + 1; m++) fo[m] = xo[m] = yo[m] = zo[m] = OutT(0);
            }
            if constexpr (EXPO == 1) {
#pragma unroll
                for (int m = 0; m < 2 * l + 1; m++)
                    pt_eb = max(pt_eb, split_bits::biased_exponent(__double_as_longlong(double(fo[m]))));
            }
            store_rows(o, e.pos, 2 * l + 1, q, fo, xo, yo, zo, GRAD);
        }
        ul *= u;
    }
    if constexpr (EXPO == 1) {
        if (pt_eb > 0) atomicMax(xi.red + q, pt_eb);
    }
}

// ----------------------------------------------------------------------------------------
// The split path's evaluation in float-float arithmetic (csrc/ff.h): the same quantities and
// recurrences as eval_group, with FP64 kept for the geometry (d, r^2, 1/r) and the radial
// coordinate t (segment choice and log1p), converted once; everything that follows (the
// solid-harmonic recurrence, the spline, the products) runs on the FP32 pipe with ~48-bit
// significands. Results are stored as float-float pairs (FF2). Points within kNearNucleus of
// the atom, and atoms with functions of l >= 5, take eval_group in FP64 instead.
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ ffa::F ff_zero() { return ffa::F{0.0f, 0.0f}; }
__device__ __forceinline__ ffa::F ff_of(float h) { return ffa::F{h, 0.0f}; }

// A rational constant a / b (small integers) as a float-float: folded by the compiler once the
// loops over l and m are unrolled.
__device__ __forceinline__ ffa::F ff_ratio(int a, int b) {
    const double c = (double)a / (double)b;
    const float h = (float)c;
    return ffa::F{h, (float)(c - (double)h)};
}

// Biased FP64 exponent of an upper bound of |v| (0: v is taken as zero): the exponent of v.h,
// plus one when v.h's significand is within 2^-15 of 2 (v.l may then carry |v| into the next
// binade). Subnormal v.h (|v| < 2^-126) counts as zero.
__device__ __forceinline__ int ff_bound_eb(ffa::F v) {
    const int b = __float_as_int(v.h) & 0x7FFFFFFF;
    const int e = b >> 23;
    if (e == 0) return 0;
    return e + 896 + ((b & 0x7FFFFF) >= 0x7FFF00 ? 1 : 0);
}

template <typename OutT>
__device__ __forceinline__ OutT ff_out(ffa::F v) {
    if constexpr (std::is_same<OutT, FF2>::value) return FF2(v);
    else return OutT(ffa::to_double(v));
}

template <int LMAX, bool GRAD, typename OutT, int EXPO>
__device__ __noinline__ void eval_group_ff(const DevSystem &s, const AtomGroup &ag, double dx, double dy, double dz,
                                          double r2, double r, double ur, const EvalOut<OutT> &o, int q, ExpoIn xi) {
    using ffa::F;
    // radial coordinate in FP64, as eval_group<double>
    const double rr = fmax(r, s.r0);
    const float sa = __logf((float)rr * (float)__ldg(s.inv_rk)) * (float)s.inv_delta;
    int k = (int)floorf(sa);
    k = k < 0 ? 0 : (k > s.n_rgrid - 2 ? s.n_rgrid - 2 : k);
    double xr = fma(rr, __ldg(s.inv_rk + k), -1.0);
    if (xr < 0.0 && k > 0) {
        k--;
        xr = fma(rr, __ldg(s.inv_rk + k), -1.0);
    } else if (xr >= s.step_m1 && k < s.n_rgrid - 2) {
        k++;
        xr = fma(rr, __ldg(s.inv_rk + k), -1.0);
    }
    const F t = ffa::from_double(log1p_small(xr, s.step_m1) * s.inv_delta);
    const F dr_scale = ffa::from_double(s.inv_delta * (r < s.r0 ? __ldg(s.inv_rk) : ur));
    const F u = ffa::from_double(ur);
    const F x = ffa::from_double(dx), y = ffa::from_double(dy), z = ffa::from_double(dz);
    const F qq = ffa::from_double(r2);
    const F x2 = ffa::twice(x), y2 = ffa::twice(y), z2 = ffa::twice(z);
    // A_m + i B_m = (x + i y)^m
    F A[LMAX + 1], B[LMAX + 1];
    A[0] = ff_of(1.0f);
    B[0] = ff_zero();
#pragma unroll
    for (int m = 1; m <= LMAX; m++) {
        if (m == 1) {
            A[1] = x;
            B[1] = y;
        } else {
            A[m] = ffa::dot2(x, A[m - 1], ffa::neg(y), B[m - 1]);
            B[m] = ffa::dot2(x, B[m - 1], y, A[m - 1]);
        }
    }
    // Pi_{l-1}^m (c) and Pi_{l-2}^m (p) with their z and r^2 derivatives (see eval_group)
    F Pc[LMAX + 1], Pcz[LMAX + 1], Pcq[LMAX + 1], Pp[LMAX + 1], Ppz[LMAX + 1], Ppq[LMAX + 1];
#pragma unroll
    for (int m = 0; m <= LMAX; m++) Pc[m] = Pcz[m] = Pcq[m] = Pp[m] = Ppz[m] = Ppq[m] = ff_zero();
    int ri = ag.r0;
    const int re = ag.r0 + ag.nr;
    int pt_eb = 0;
    F ul = ff_of(1.0f);  // u^l
#pragma unroll
    for (int l = 0; l <= LMAX; l++) {
        F S[2 * LMAX + 1], Gx[2 * LMAX + 1], Gy[2 * LMAX + 1], Gz[2 * LMAX + 1];
        bool zx[2 * LMAX + 1], zy[2 * LMAX + 1], zz[2 * LMAX + 1];
#pragma unroll
        for (int m = 0; m <= l; m++) {
            F p, pz = ff_zero(), pq = ff_zero();
            const bool zpz = (m == l), zpq = (l - m < 2);
            if (m == l) {
                p = ff_of((float)double_factorial_odd(m));  // an odd integer below 2^24: exact
            } else if (m == l - 1) {
                p = ffa::mulf(ffa::mul(z, Pc[m]), (float)(2 * m + 1));
                pz = ffa::mulf(Pc[m], (float)(2 * m + 1));
            } else {
                const F c1 = ff_ratio(2 * l - 1, l - m), c2 = ff_ratio(l + m - 1, l - m);
                const F nc2 = ffa::neg(c2);
                p = ffa::dot2(c1, ffa::mul(z, Pc[m]), nc2, ffa::mul(qq, Pp[m]));
                pz = ffa::mul(c1, ffa::fma(z, Pcz[m], Pc[m]));
                if (l - 2 != m) pz = ffa::fma(nc2, ffa::mul(qq, Ppz[m]), pz);
                const F pq_p = (l - 2 - m >= 2) ? ffa::fma(qq, Ppq[m], Pp[m]) : Pp[m];
                pq = (l - 1 - m >= 2) ? ffa::dot2(c1, ffa::mul(z, Pcq[m]), nc2, pq_p) : ffa::mul(nc2, pq_p);
            }
            Pp[m] = Pc[m]; Ppz[m] = Pcz[m]; Ppq[m] = Pcq[m];
            Pc[m] = p; Pcz[m] = pz; Pcq[m] = pq;
            const F kn = ffa::F{s.knorm_h[l][m], s.knorm_l[l][m]};
            const F kp = ffa::mul(kn, p);
            const F kpq = zpq ? ff_zero() : ffa::mul(kn, pq);
            const F kdx = zpq ? ff_zero() : ffa::mul(x2, kpq), kdy = zpq ? ff_zero() : ffa::mul(y2, kpq);
            const F kdz = zpz ? (zpq ? ff_zero() : ffa::mul(z2, kpq))
                              : (zpq ? ffa::mul(kn, pz) : ffa::fma(z2, kpq, ffa::mul(kn, pz)));
            const bool zdz = zpz && zpq;
            if (m == 0) {
                S[l] = kp;
                Gx[l] = kdx;
                Gy[l] = kdy;
                Gz[l] = kdz;
                zx[l] = zy[l] = zpq;
                zz[l] = zdz;
            } else {
                const F kpf = ffa::mulf(kp, (float)m);
                S[l + m] = ffa::mul(kp, A[m]);
                Gx[l + m] = zpq ? ffa::mul(kpf, A[m - 1]) : ffa::dot2(kdx, A[m], kpf, A[m - 1]);
                Gy[l + m] = m == 1 ? (zpq ? ff_zero() : ffa::mul(kdy, A[m]))
                                   : (zpq ? ffa::neg(ffa::mul(kpf, B[m - 1])) : ffa::dot2(kdy, A[m], ffa::neg(kpf), B[m - 1]));
                Gz[l + m] = zdz ? ff_zero() : ffa::mul(kdz, A[m]);
                S[l - m] = ffa::mul(kp, B[m]);
                Gx[l - m] = m == 1 ? (zpq ? ff_zero() : ffa::mul(kdx, B[m]))
                                   : (zpq ? ffa::mul(kpf, B[m - 1]) : ffa::dot2(kdx, B[m], kpf, B[m - 1]));
                Gy[l - m] = zpq ? ffa::mul(kpf, A[m - 1]) : ffa::dot2(kdy, B[m], kpf, A[m - 1]);
                Gz[l - m] = zdz ? ff_zero() : ffa::mul(kdz, B[m]);
                zx[l + m] = false;
                zy[l + m] = (m == 1 && zpq);
                zz[l + m] = zz[l - m] = zdz;
                zx[l - m] = (m == 1 && zpq);
                zy[l - m] = false;
            }
        }
        const F ulu = ffa::mul(ul, u);                       // u^(l+1)
        const F a_dr = ffa::mul(dr_scale, ulu);               // dR/ds -> g'(r)/r
        const F a_r = ffa::mulf(ffa::mul(u, ulu), (float)l);  // R -> the l R / r part of g'(r)/r
        for (; ri < re; ri++) {
            const RfnEntry e = s.rfn[ri];
            if (e.l != l) break;
            OutT fo[2 * LMAX + 1], xo[2 * LMAX + 1], yo[2 * LMAX + 1], zo[2 * LMAX + 1];
            if (r < s.fn_rc[e.fn]) {
                const size_t seg = (size_t)e.fn * (s.n_rgrid - 1) + k;
                const float4 ch = __ldg(reinterpret_cast<const float4 *>(s.coef_f32 + seg * 4));
                const float4 cl = __ldg(reinterpret_cast<const float4 *>(s.coef_lo + seg * 4));
                const F c0{ch.x, cl.x}, c1{ch.y, cl.y}, c2{ch.z, cl.z}, c3{ch.w, cl.w};
                // R = c0 + t (c1 + t a), dR/dt = c1 + t (2 a + c3 t), a = c2 + c3 t
                const F a = ffa::fma(c3, t, c2);
                const F R = ffa::fma(ffa::fma(a, t, c1), t, c0);
                const F dRds = ffa::fma(ffa::fma(c3, t, ffa::twice(a)), t, c1);
                const F g = ffa::mul(R, ul);
                const F gpu = l == 0 ? ffa::mul(dRds, a_dr) : ffa::dot2(dRds, a_dr, ffa::neg(R), a_r);
                const F gx = ffa::mul(gpu, x), gy = ffa::mul(gpu, y), gz = ffa::mul(gpu, z);
#pragma unroll
                for (int m = 0; m < 2 * l + 1; m++) {
                    const F fv = ffa::mul(g, S[m]);
                    if constexpr (EXPO == 1) pt_eb = max(pt_eb, ff_bound_eb(fv));
                    fo[m] = ff_out<OutT>(fv);
                    if (GRAD) {
                        xo[m] = ff_out<OutT>(zx[m] ? ffa::mul(gx, S[m]) : ffa::dot2(gx, S[m], g, Gx[m]));
                        yo[m] = ff_out<OutT>(zy[m] ? ffa::mul(gy, S[m]) : ffa::dot2(gy, S[m], g, Gy[m]));
                        zo[m] = ff_out<OutT>(zz[m] ? ffa::mul(gz, S[m]) : ffa::dot2(gz, S[m], g, Gz[m]));
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < 2 * l + 1; m++) fo[m] = xo[m] = yo[m] = zo[m] = OutT(0);
            }
            store_rows(o, e.pos, 2 * l + 1, q, fo, xo, yo, zo, GRAD);
        }
        ul = ffa::mul(ul, u);
    }
    if constexpr (EXPO == 1) {
        if (pt_eb > 0) atomicMax(xi.red + q, pt_eb);
    }
}

// Arithmetic of the split path's evaluation: float-float (eval_group_ff), stored as FF2.
struct FFTag {};
template <typename T>
struct out_of {
    using type = T;
};
template <>
struct out_of<FFTag> {
    using type = FF2;
};

template <int LMAX, bool GRAD, typename T, int EXPO, typename OutT>
__device__ __forceinline__ void eval_group_dispatch(const DevSystem &s, const AtomGroup &ag, double dx, double dy,
                                                    double dz, double r2, double r, double ur, const EvalOut<OutT> &o, int q,
                                                    const ExpoIn &xi) {
    if constexpr (std::is_same<T, FFTag>::value) {
        // float-float up to l = 4; atoms with g functions and beyond, and points near a nucleus,
        // in FP64 (instantiating the float-float code for l = 5, 6 would take the kernels' stack
        // frames above 1 KB)
        if (LMAX > 4 || r < kNearNucleus)
            eval_group<LMAX, double, GRAD, OutT, EXPO>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi);
        else
            eval_group_ff<LMAX < 4 ? LMAX : 4, GRAD, OutT, EXPO>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi);
    } else if constexpr (EXPO != 0 || std::is_same<T, double>::value)
        eval_group<LMAX, double, GRAD, OutT, EXPO>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi);
    else if (r < kNearNucleus)
        eval_group<LMAX, double, GRAD, OutT, 0>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi);
    else
        eval_group<LMAX, float, GRAD, OutT, 0>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi);
}

template <bool GRAD, typename T, int EXPO, typename OutT>
__device__ __forceinline__ void eval_batch(const DevSystem &s, int b, const EvalOut<OutT> &o, int *red = nullptr) {
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int g0 = s.agrp_off[b], ng = s.agrp_off[b + 1] - g0;
    const int qmax = o.qmax;
    const int total = ng * qmax;
    const ExpoIn xi{red};
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int gl = idx / qmax, q = idx - gl * qmax;
        const AtomGroup ag = s.agrp[g0 + gl];
        if (q >= P) {  // padding points: zero rows
            OutT z0[2 * NAO_LMAX + 1];
#pragma unroll
            for (int m = 0; m < 2 * NAO_LMAX + 1; m++) z0[m] = OutT(0);
            for (int ri = ag.r0; ri < ag.r0 + ag.nr; ri++) {
                const RfnEntry e = s.rfn[ri];
                store_rows(o, e.pos, 2 * e.l + 1, q, z0, z0, z0, z0, GRAD);
            }
            continue;
        }
        const int p = p0 + q;
        const double dx = __dsub_rn(s.px[p], s.atom_xyz[3 * ag.atom]);
        const double dy = __dsub_rn(s.py[p], s.atom_xyz[3 * ag.atom + 1]);
        const double dz = __dsub_rn(s.pz[p], s.atom_xyz[3 * ag.atom + 2]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        // 1/r from the library's reciprocal square root (about one ulp) and r = r^2 (1/r): one
        // FP64 function instead of a square root and a division
        const double ur = rsqrt(r2);
        const double r = r2 > 0.0 ? r2 * ur : 0.0;
        switch (ag.lmax) {
            case 0: eval_group_dispatch<0, GRAD, T, EXPO>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi); break;
            case 1: eval_group_dispatch<1, GRAD, T, EXPO>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi); break;
            case 2: eval_group_dispatch<2, GRAD, T, EXPO>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi); break;
            case 3: eval_group_dispatch<3, GRAD, T, EXPO>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi); break;
            case 4: eval_group_dispatch<4, GRAD, T, EXPO>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi); break;
            case 5: eval_group_dispatch<5, GRAD, T, EXPO>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi); break;
            default: eval_group_dispatch<6, GRAD, T, EXPO>(s, ag, dx, dy, dz, r2, r, ur, o, q, xi); break;
        }
    }
}

template <bool GRAD, typename T>
__device__ __forceinline__ EvalOut<T> batch_out(const DevSystem &s, int b, int Ppad, T *scratch) {
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
    return o;
}

// One CTA per batch; the batch's block of scratch holds, per reduced-basis row j,
// [phi | d/dx | d/dy | d/dz] over Ppad points each (GRAD) or phi alone, in type T.
template <bool GRAD, typename T>
__global__ void __launch_bounds__(256) eval_chunk_kernel(DevSystem s, int32_t b0, typename out_of<T>::type *scratch) {
    using OutT = typename out_of<T>::type;
    const int b = b0 + blockIdx.x;
    const int P = s.batch_off[b + 1] - s.batch_off[b];
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    eval_batch<GRAD, T, 0>(s, b, batch_out<GRAD, OutT>(s, b, Ppad, scratch));
}

// The density's evaluation on the split path (float-float, FF2 values): as eval_chunk_kernel,
// and the point exponents of the slicing: expo[batch_off[b] + q] = the exponent of point q, from
// the binade of an upper bound of max_i |phi_iq| (split_bits::exponent_of_binade). Dynamic shared
// memory: n_red >= P_b ints.
template <bool GRAD>
__global__ void __launch_bounds__(256) eval_split_kernel(DevSystem s, int32_t b0, FF2 *scratch, int32_t *expo,
                                                         int n_red) {
    extern __shared__ int red_sh[];
    const int b = b0 + blockIdx.x;
    const int p0 = s.batch_off[b], P = s.batch_off[b + 1] - p0;
    const int Ppad = (P + NAO_PPAD - 1) & ~(NAO_PPAD - 1);
    for (int i = threadIdx.x; i < n_red; i += blockDim.x) red_sh[i] = 0;
    __syncthreads();
    eval_batch<GRAD, FFTag, 1>(s, b, batch_out<GRAD, FF2>(s, b, Ppad, scratch), red_sh);
    __syncthreads();
    for (int q = threadIdx.x; q < P; q += blockDim.x) expo[p0 + q] = split_bits::exponent_of_binade(red_sh[q]);
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
    eval_batch<GRAD, T, 0>(s, b, o);
}

}  // namespace

cudaError_t launch_relevance_minr2(const double *atom_xyz, const int32_t *bmol, const int32_t *aoff, int32_t max_atoms,
                                   const double *px, const double *py, const double *pz, const int32_t *batch_off,
                                   int64_t n_batches, double *minr2, cudaStream_t st) {
    if (n_batches <= 0) return cudaSuccess;
    minr2_kernel<<<(unsigned)n_batches, 256, 0, st>>>(atom_xyz, bmol, aoff, max_atoms, px, py, pz, batch_off, minr2);
    return cudaGetLastError();
}

cudaError_t launch_eval(const DevSystem &s, int32_t b0, int32_t b1, nao_precision prec, bool grad, double *scratch,
                        cudaStream_t st) {
    if (b1 <= b0) return cudaSuccess;
    if (prec == NAO_FP32) {
        float *f = reinterpret_cast<float *>(scratch);
        if (grad) eval_chunk_kernel<true, float><<<b1 - b0, 256, 0, st>>>(s, b0, f);
        else eval_chunk_kernel<false, float><<<b1 - b0, 256, 0, st>>>(s, b0, f);
    } else if (prec == NAO_SPLIT) {
        FF2 *f = reinterpret_cast<FF2 *>(scratch);
        if (grad) eval_chunk_kernel<true, FFTag><<<b1 - b0, 256, 0, st>>>(s, b0, f);
        else eval_chunk_kernel<false, FFTag><<<b1 - b0, 256, 0, st>>>(s, b0, f);
    } else {
        if (grad) eval_chunk_kernel<true, double><<<b1 - b0, 256, 0, st>>>(s, b0, scratch);
        else eval_chunk_kernel<false, double><<<b1 - b0, 256, 0, st>>>(s, b0, scratch);
    }
    return cudaGetLastError();
}

cudaError_t launch_eval_split(const DevSystem &s, int32_t b0, int32_t b1, bool grad, double *scratch, int32_t *expo,
                              int32_t n_red, cudaStream_t st) {
    if (b1 <= b0) return cudaSuccess;
    const size_t smem = (size_t)n_red * 4;
    FF2 *f = reinterpret_cast<FF2 *>(scratch);
    if (grad) eval_split_kernel<true><<<b1 - b0, 256, smem, st>>>(s, b0, f, expo, n_red);
    else eval_split_kernel<false><<<b1 - b0, 256, smem, st>>>(s, b0, f, expo, n_red);
    return cudaGetLastError();
}

cudaError_t launch_eval_one(const DevSystem &s, int32_t b, nao_precision prec, double *phi, double *grad,
                            cudaStream_t st) {
    if (prec == NAO_FP32) {
        if (grad) eval_export_kernel<true, float><<<1, 256, 0, st>>>(s, b, phi, grad);
        else eval_export_kernel<false, float><<<1, 256, 0, st>>>(s, b, phi, nullptr);
    } else if (prec == NAO_SPLIT) {
        if (grad) eval_export_kernel<true, FFTag><<<1, 256, 0, st>>>(s, b, phi, grad);
        else eval_export_kernel<false, FFTag><<<1, 256, 0, st>>>(s, b, phi, nullptr);
    } else {
        if (grad) eval_export_kernel<true, double><<<1, 256, 0, st>>>(s, b, phi, grad);
        else eval_export_kernel<false, double><<<1, 256, 0, st>>>(s, b, phi, nullptr);
    }
    return cudaGetLastError();
}

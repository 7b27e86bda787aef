/*
 * nao.h -- C ABI of the GB300 real-space grid-integration library (libnao.so).
 *
 * The library integrates, on one GPU, the two real-space operations of an all-electron
 * Kohn-Sham code with numeric atom-centred orbitals (Huhn et al., "GPGPU Acceleration of
 * All-Electron Electronic Structure Theory Using Localized Numeric Atom-Centered Basis
 * Functions", arXiv:1912.06636):
 *
 *   Hamiltonian  h_ij = sum_r w(r) [ phi_i(r) v(r) phi_j(r) + 1/2 grad phi_i . grad phi_j ]
 *                (Eq. H_int_aims with the kinetic operator written in its symmetric form;
 *                 Eqs. H_decomp / H_contrib_batch split it over batches of points)
 *   Density      n(r) = sum_ij phi_i(r) n_ij phi_j(r)          (Eq. Density)
 *
 * where phi_i(r) = R_f(|r - R_A|) Y_lm(r^) is basis function i (atom A, radial function f
 * of A's species, m), R_f a cubic spline through a tabulated radial function that is zero
 * beyond its cutoff (Sec. 3.2.1), and Y_lm a real spherical harmonic.
 *
 * Conventions for every call:
 *   - Status codes; nothing aborts, traps or throws across the ABI.
 *   - "_dev" pointers are CUDA device pointers on the handle's device; "host" pointers are
 *     ordinary host memory. The caller owns every buffer it passes in and keeps it alive
 *     until the work on the given stream has completed. The library owns the handle and
 *     the device tables and scratch it allocated at create time, and frees them in
 *     nao_destroy.
 *   - Work is enqueued asynchronously on the CUDA stream passed in (cudaStream_t as void*,
 *     NULL = the legacy default stream). A handle serves one stream at a time: calls on
 *     the same handle must not overlap on the GPU.
 *   - Device-side failures (a kernel's own bounds or timeout check) are recorded in the
 *     handle and reported by nao_sync_status and by the next call on the handle.
 *   - There is no CPU fallback: every numeric step runs in the library's CUDA kernels.
 */
#ifndef NAO_H
#define NAO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nao_grid nao_grid; /* opaque, library-owned */

typedef enum {
    NAO_OK = 0,
    NAO_ERR_INVALID_ARG = 1,   /* a bad pointer, size, index, non-finite value or option */
    NAO_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation failed */
    NAO_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
    NAO_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up */
    NAO_ERR_INTERNAL = 5,      /* a device-side consistency check failed */
    NAO_ERR_UNSUPPORTED = 6    /* valid request the build or device cannot serve */
} nao_status;

/* Arithmetic of the contractions (Eq. batch_matrix_mult and the density analogue).
 *   NAO_FP64  : FP64 everywhere.
 *   NAO_FP32  : basis functions and contractions in FP32 (FP64 inside 0.1 bohr of a
 *               nucleus), per-batch results accumulated into H / n in FP64.
 *   NAO_SPLIT : basis functions evaluated in float-float arithmetic (about 48 significant
 *               bits; FP64 inside 0.1 bohr of a nucleus and for l >= 5), cut into integer
 *               slices (Ozaki splitting; bf16 or e4m3 digits, options.split_digits); the
 *               slice products run on the tcgen05 tensor cores with exact FP32 accumulation
 *               and are recombined as 64-bit integers, then scaled into FP64.            */
typedef enum { NAO_FP64 = 0, NAO_FP32 = 1, NAO_SPLIT = 2 } nao_precision;

/* Terms of nao_integrate_h. The overlap s_ij (Eq. OverlapNoPeriodic) is
 * NAO_TERM_POTENTIAL with v_dev == NULL (v = 1): the paper integrates it with the same
 * code as h (Sec. 3.2.1).                                                                */
enum { NAO_TERM_POTENTIAL = 1u, NAO_TERM_KINETIC = 2u, NAO_TERM_TAU = 4u /* nao_integrate_h_tau only */ };

/* The system, exactly as the paper states the problem (Sec. 3.2.1, Sec. 3.3):
 * atoms with species; per species a list of radial functions (angular momentum l and a
 * cutoff radius); each radial function tabulated on the logarithmic grid
 * r_k = r0 (r_last/r0)^(k/(n_rgrid-1)); and the integration points with their weights.
 * All pointers are HOST pointers, read during nao_grid_create only.
 * Basis order: atom, then the species' radial functions in order, then m = -l..l.         */
typedef struct {
    int32_t n_atoms;
    const double *atom_xyz;          /* [n_atoms*3] bohr */
    const int32_t *atom_species;     /* [n_atoms], 0..n_species-1 */
    int32_t n_species;
    const int32_t *species_fn_offset; /* [n_species+1] radial functions of species s are
                                         species_fn_offset[s] .. species_fn_offset[s+1]-1 */
    const int32_t *fn_l;             /* [n_fn] angular momentum 0..6 */
    const double *fn_cutoff;         /* [n_fn] bohr, 0 < cutoff <= r_last; R_f = 0 beyond */
    int32_t n_rgrid;                 /* >= 4 */
    double r0, r_last;               /* 0 < r0 < r_last */
    const double *fn_table;          /* [n_fn*n_rgrid] R_f(r_k) (the radial function itself) */
    int64_t n_points;                /* >= 1, < 2^31 */
    const double *pt_xyz;            /* [n_points*3] bohr; no point may coincide with a nucleus */
    const double *pt_w;              /* [n_points] integration weights (finite) */
} nao_system_desc;

typedef struct {
    int32_t max_batch_points; /* target batch size B (Sec. 3.3.1; the paper uses 200 on GPUs); default 200 */
    int32_t split_slices;     /* slices per operand on the NAO_SPLIT path: 4..12 with bf16 digits
                                 (default 12), 8..16 with e4m3 digits (split_digits). Each bf16
                                 slice adds 6 bits and each e4m3 slice 5: the error of an element
                                 falls about 64x (32x) per slice (measured e_H on an 8-atom cell
                                 with 20 radial shells: 1.6e-9 at 10, 4.6e-11 at 11, 8.6e-13 at 12
                                 bf16 slices). bf16 with 4..10 slices runs 128x48 tensor-core
                                 tiles, otherwise 128x32. */
    int32_t deterministic;    /* 0 (default): the batches' contributions to H are FP64 atomic
                                 additions, whose order (and so H's last bits) varies from run to
                                 run. 1: every contribution is added exactly as a 128-bit
                                 fixed-point integer (resolution 2^-90, contributions below 2^37)
                                 and H is converted once at the end, so H is bitwise the same
                                 from run to run on every precision path (each contribution is
                                 rounded to 2^-90, the exact sum converted with a relative error
                                 below 2^-52); costs 16 bytes of device memory per H
                                 element of every system, taken at create, and two integer atomics
                                 per contribution. n, grad n, the Hessian and N_e have no atomics
                                 and are reproducible either way; the Pulay matrices and the Bloch
                                 sum keep FP64 atomics. */
    int32_t device;           /* CUDA device ordinal; -1 = the calling thread's current device */
    int64_t scratch_bytes;    /* device scratch for evaluated basis functions; 0 = library default (8 GiB;
                                 the split path's slices take three times this). Memory is taken only
                                 up to what the batches need; smaller values mean more, smaller launches */
    int32_t capture_graph;    /* 1: the first call of each (operation, precision, terms) records
                                 its kernel launches as a CUDA graph on a stream the handle
                                 owns; later calls upload that call's pointer tables and replay
                                 the graph, ordered after the caller's stream's earlier work and
                                 before its later work (events). Not used while profiling.
                                 Default 0 (plain launches on the caller's stream). */
    int32_t autotune;         /* 1 (default): the first NAO_SPLIT Hamiltonian call times 128x48 against
                                 128x32 tensor-core tiles for each (N_b, P_b) bucket of the batch-size
                                 histogram (nao_get_tuning reports the result); 0: a fixed rule (48
                                 where S <= 10, else 32). */
    int32_t split_digits;     /* digit format of the NAO_SPLIT path: 0 (default) balanced base-64
                                 digits stored as bf16 (kind::f16 MMAs); 1 balanced base-32 digits
                                 stored as e4m3 (every integer |d| <= 16 is exact in e4m3;
                                 kind::f8f6f4 MMAs at twice the bf16 rate, half the bytes per
                                 digit). 14 e4m3 slices carry 70 bits, 11 bf16 slices 66. */
} nao_options;

typedef struct {
    int64_t n_basis;          /* nb: H and P are nb x nb, row-major */
    int64_t n_points;
    int64_t n_batches;
    int64_t rel_total;        /* sum over batches of |nnz(B)| */
    int32_t max_batch_points; /* largest |B| */
    int32_t max_batch_basis;  /* largest |nnz(B)| */
    int64_t device_bytes;     /* device memory held by the handle */
    int64_t flops_h;          /* algorithmic FLOPs of one nao_integrate_h: sum_b 4 P_b N_b (N_b+1) */
    int64_t flops_n;          /* algorithmic FLOPs of one nao_update_density: sum_b 2 P_b N_b^2 + 2 P_b N_b */
    int32_t n_systems;        /* systems of the handle (1 for nao_grid_create) */
    int32_t n_atoms;          /* atoms of the handle (all systems); F of nao_pulay_forces is 3 x this */
} nao_grid_info;

/* Fill *opts with the defaults above. */
nao_status nao_default_options(nao_options *opts);

/* Build a handle (Sec. 3.3.1-3.3.2): partition the points into batches by recursive
 * bisection (the batch-partition rule below), find each batch's reduced basis nnz(B)
 * (the relevance rule below), fit the radial splines, and upload everything to the device.
 *   Batch-partition rule: split(S) with n = |S| and k = ceil(n/B); if k <= 1, S is a batch
 *     (points kept in their current order); otherwise cut along the axis of largest
 *     bounding-box extent (ties x < y < z), ordering S by (coordinate, point index), the
 *     first floor(n*floor(k/2)/k) points going left; recurse left, then right.
 *   Relevance rule: (A, f, m) is in nnz(B) iff some point of B has
 *     (dx*dx + dy*dy) + dz*dz < rc_f*rc_f in separately rounded FP64 operations.
 * desc, opts: host pointers (opts may be NULL for defaults). On success *out holds the new
 * handle; on failure *out is set to NULL and nothing is leaked.
 * Errors: NAO_ERR_INVALID_ARG (see nao_system_desc), NAO_ERR_OUT_OF_MEMORY, NAO_ERR_CUDA. */
nao_status nao_grid_create(const nao_system_desc *desc, const nao_options *opts, nao_grid **out);

/* One handle over several independent systems (molecules) that share the logarithmic
 * radial grid (n_rgrid, r0, r_last): each system is partitioned into its own batches
 * (no batch mixes systems), and one launch of each kernel covers the batches of all of
 * them, so many small molecules fill the GPU together (the batch loop of Sec. 3.3 runs
 * over the union of their batches). Global numbering: basis functions, points and atoms
 * of system m follow those of systems 0..m-1; nao_get_info, nao_export_batches and
 * nao_evaluate_batch use it. descs: host array [n_systems], each as for nao_grid_create;
 * n_systems >= 1. max_batch_points: host array [n_systems] of per-system batch sizes B
 * (1..1024), or NULL for options.max_batch_points everywhere. The single-system calls
 * (nao_integrate_h, nao_update_density and their host and noalloc forms) require
 * n_systems == 1; use the _many forms otherwise.
 * Errors: as nao_grid_create; NAO_ERR_INVALID_ARG if the radial grids differ.              */
nao_status nao_grid_create_many(const nao_system_desc *descs, int32_t n_systems, const int32_t *max_batch_points,
                                const nao_options *opts, nao_grid **out);

/* Basis and point ranges of system m in the global numbering: basis functions
 * basis_offset .. basis_offset+n_basis-1, points point_offset .. point_offset+n_points-1,
 * batches batch_begin .. batch_end-1. Any output pointer may be NULL.                      */
nao_status nao_get_system(const nao_grid *g, int32_t m, int64_t *basis_offset, int64_t *n_basis,
                          int64_t *point_offset, int64_t *n_points, int64_t *batch_begin, int64_t *batch_end);

/* Split-path tile width chosen for every batch (host array [n_batches]; 48 or 32, 0 before the
 * first NAO_SPLIT call) and the number of histogram buckets the autotuner timed (-1 while
 * tuning is pending). Either pointer may be NULL.                                            */
nao_status nao_get_tuning(const nao_grid *g, int32_t *tile_width, int32_t *buckets_timed);

/* Release the handle and all its device memory. NULL-safe. Synchronises the device work
 * the handle has enqueued before freeing.                                                */
nao_status nao_destroy(nao_grid *g);

/* Sizes and algorithmic work counts of the handle. */
nao_status nao_get_info(const nao_grid *g, nao_grid_info *info);

/* Copy the partition and the reduced bases to caller-allocated HOST arrays:
 * batch_offsets[n_batches+1], point_perm[n_points] (original index of each batch-ordered
 * point), rel_offsets[n_batches+1], rel_idx[rel_total] (ascending global basis indices
 * per batch). Any pointer may be NULL to skip that array.                                 */
nao_status nao_export_batches(const nao_grid *g, int64_t *batch_offsets, int64_t *point_perm,
                              int64_t *rel_offsets, int32_t *rel_idx);

/* Host-only set-up steps, without a handle or a GPU (the same code nao_grid_create runs).
 * nao_partition_points (Sec. 3.3.1): the batch-partition rule above applied to pt_xyz
 * [n_points*3] (host) with B = max_batch_points (>= 1). Outputs (host, caller-allocated):
 * batch_offsets [n_batches+1], point_perm [n_points] as nao_export_batches; *n_batches =
 * ceil(n_points/B). More batches than max_batches: NAO_ERR_INVALID_ARG with *n_batches set
 * (call again with room). Non-finite coordinates: NAO_ERR_INVALID_ARG.
 * nao_radial_spline (Sec. 3.2.1, the NAO radial functions, represented as cubic splines through
 * their tables as in nao_grid_create): the natural cubic spline in
 * the index coordinate s = ln(r/r0)/Delta through (k, fn_table[k]), k = 0..n_rgrid-1 (>= 4),
 * as coef [(n_rgrid-1)*4] (host): on segment k, R = c0 + c1 t + c2 t^2 + c3 t^3 with t = s - k,
 * c = coef + 4k. Non-finite table entries: NAO_ERR_INVALID_ARG.                              */
nao_status nao_partition_points(const double *pt_xyz, int64_t n_points, int64_t max_batch_points, int64_t max_batches,
                                int64_t *batch_offsets, int64_t *point_perm, int64_t *n_batches);
nao_status nao_radial_spline(const double *fn_table, int32_t n_rgrid, double *coef);

/* Hamiltonian integration (Eq. H_int_aims; Eqs. H_decomp, H_contrib_batch,
 * batch_matrix_mult): H_dev[i*nb+j] = sum_p w_p [ phi_i v_p phi_j (if POTENTIAL)
 *                                              + 1/2 grad phi_i . grad phi_j (if KINETIC) ].
 * v_dev: device [n_points] in the caller's original point order, or NULL for v = 1.
 * H_dev: device [nb*nb] row-major, overwritten (both triangles; exactly symmetric).
 * terms: a non-empty subset of NAO_TERM_POTENTIAL | NAO_TERM_KINETIC.
 * Errors: NAO_ERR_INVALID_ARG (NULL handle/H, bad terms or precision), NAO_ERR_CUDA,
 * NAO_ERR_UNSUPPORTED (precision not built for this device).                               */
nao_status nao_integrate_h(nao_grid *g, const double *v_dev, uint32_t terms, nao_precision prec,
                           double *H_dev, void *cuda_stream);

/* The same with the meta-GGA term (the part of the exchange-correlation potential that depends on
 * the kinetic-energy density tau, Sec. 3.4's "extra weighted" gradient product): with
 * NAO_TERM_TAU in terms, H_dev additionally receives sum_p w_p v_tau,p 1/2 grad phi_i . grad phi_j.
 * It enters as a weight on the three gradient columns (w (kappa + v_tau) / 2, kappa = 1 with
 * NAO_TERM_KINETIC), so it costs no extra contraction. vtau_dev: device [n_points], original
 * point order; required (non-NULL) with NAO_TERM_TAU. terms: a non-empty subset of
 * NAO_TERM_POTENTIAL | NAO_TERM_KINETIC | NAO_TERM_TAU. All three precisions; single-system
 * handles (grouped: NAO_ERR_INVALID_ARG). Other arguments and errors as nao_integrate_h.    */
nao_status nao_integrate_h_tau(nao_grid *g, const double *v_dev, const double *vtau_dev, uint32_t terms,
                               nao_precision prec, double *H_dev, void *cuda_stream);

/* Density update (Eq. Density, Sec. 3.3.5): n_dev[p] = sum_ij phi_i(r_p) P_ij phi_j(r_p)
 * for every point p (original order; 0 for points in batches without basis functions),
 * and, if n_electrons_dev is not NULL, n_electrons_dev[0] = sum_p w_p n_p (FP64).
 * P_dev: device [nb*nb] row-major, symmetric (only the upper triangle P[i][j], i <= j, is
 * read). n_dev: device [n_points]. n_electrons_dev: device [1] or NULL.                    */
nao_status nao_update_density(nao_grid *g, const double *P_dev, nao_precision prec, double *n_dev,
                              double *n_electrons_dev, void *cuda_stream);

/* Grouped forms: the same operations for every system of the handle in one pass of the
 * kernels (one launch per kernel for all systems). Arrays are HOST arrays of n_systems
 * DEVICE pointers, read during the call; entry m refers to system m in its own numbering
 * (H_dev[m] is n_basis(m) x n_basis(m), v_dev[m] and n_dev[m] have n_points(m) entries in
 * system m's original point order).
 *   nao_integrate_h_many: v_dev may be NULL (v = 1 for every system), or an array whose
 *     NULL entries mean v = 1 for that system; every H_dev[m] is required.
 *   nao_update_density_many: every P_dev[m] and n_dev[m] is required; n_electrons_dev may
 *     be NULL, or an array whose non-NULL entries receive sum_p w_p n_p of that system.
 * Errors: as the single-system forms.                                                      */
nao_status nao_integrate_h_many(nao_grid *g, const double *const *v_dev, uint32_t terms, nao_precision prec,
                                double *const *H_dev, void *cuda_stream);
nao_status nao_update_density_many(nao_grid *g, const double *const *P_dev, nao_precision prec,
                                   double *const *n_dev, double *const *n_electrons_dev, void *cuda_stream);

/* Density and its gradient (Sec. 2: the density gradients GGA functionals need, "straightforward
 * extensions of Eq. Density"; Sec. "Density and Density Derivatives"):
 *     grad n(r_p) = 2 sum_ij grad phi_i(r_p) P_ij phi_j(r_p)   (P symmetric),
 * computed with n from one product T = Phi P over all of P (no tile-pair symmetry), so one call
 * costs about twice nao_update_density plus the gradient evaluation. grad_dev: device
 * [3 * n_points], component-major (d/dx for every point, then d/dy, then d/dz), original point
 * order; n_dev and n_electrons_dev as nao_update_density. All three precisions (NAO_SPLIT
 * takes P' = P over all of K and the gradient rows of the evaluated block in its epilogue).
 * The _many form: host arrays of per-system device pointers as nao_update_density_many,
 * grad_dev[m] of 3 * n_points(m) entries.                                                      */
nao_status nao_update_density_gradient(nao_grid *g, const double *P_dev, nao_precision prec, double *n_dev,
                                       double *grad_dev, double *n_electrons_dev, void *cuda_stream);
nao_status nao_update_density_gradient_many(nao_grid *g, const double *const *P_dev, nao_precision prec,
                                            double *const *n_dev, double *const *grad_dev,
                                            double *const *n_electrons_dev, void *cuda_stream);

/* Density, gradient and Hessian (Sec. 2: the Hessian of the density, six components, needed for
 * forces and stresses):
 *     d_a d_b n(r_p) = 2 sum_ij P_ij (phi_i d_a d_b phi_j + d_a phi_i d_b phi_j)   (P symmetric),
 * from the basis functions' second derivatives and the four products Phi P, (d_a Phi) P over all
 * of P. NAO_FP64: everything in FP64; NAO_FP32: the derivatives are computed in FP64 and
 * rounded once to FP32, the products and the per-tile epilogue run in FP32 (about 1e-6 of the
 * magnitude sums); NAO_SPLIT: the derivatives in FP64, the four products as Ozaki slice products
 * on the tensor cores (the handle's slice count and digit format; four passes, P' sliced once),
 * epilogues in FP64 (about 1e-12 of the magnitude sums). hess_dev: device [6 * n_points],
 * component-major in the order xx, xy, xz, yy, yz, zz, original point order; n_dev, grad_dev and
 * n_electrons_dev as nao_update_density_gradient. Single-system handles only (grouped:
 * NAO_ERR_INVALID_ARG). A batch whose 10-row evaluation (N_b x 10 Ppad values) exceeds the
 * evaluation scratch returns NAO_ERR_UNSUPPORTED (raise scratch_bytes).                                                                              */
nao_status nao_update_density_hessian(nao_grid *g, const double *P_dev, nao_precision prec, double *n_dev,
                                      double *grad_dev, double *hess_dev, double *n_electrons_dev, void *cuda_stream);

/* Local Pulay force terms (Sec. 2: F^{P,local}_at = -2 sum_ij int [grad_at phi_i] n_ij h_KS phi_j
 * + 2 sum_ij int [grad_at phi_i] q_ij phi_j, q the energy-weighted density matrix), assembled from
 * matrix elements with basis-function indices as the paper describes for forces:
 *     M_dev[c*nb*nb + i*nb + j] = sum_p w_p d_c phi_i(r_p) (-1/2 lap + v_p) phi_j(r_p),
 *     S_dev[c*nb*nb + i*nb + j] = sum_p w_p d_c phi_i(r_p) phi_j(r_p),        c = x, y, z,
 * (not symmetric; both overwritten) from the basis functions' second derivatives, in FP64
 * (NAO_FP64) or with the derivatives rounded once to FP32 and the products in FP32 (NAO_FP32;
 * NAO_SPLIT: NAO_ERR_UNSUPPORTED). v_dev: device [n_points] original order, or NULL for v = 1.
 * Single-system handles; scratch rules as nao_update_density_hessian.
 * nao_pulay_forces: F_dev[3*a + c] = 2 sum_{i on atom a} sum_j (n_ij M^c_ij - q_ij S^c_ij)
 * (grad_at phi_i = -grad phi_i for a function on atom a), n_dev and q_dev device [nb*nb]
 * row-major, F_dev device [3*n_atoms], overwritten.                                            */
nao_status nao_pulay_matrices(nao_grid *g, const double *v_dev, nao_precision prec, double *M_dev, double *S_dev,
                              void *cuda_stream);
nao_status nao_pulay_forces(nao_grid *g, const double *n_dev, const double *q_dev, const double *M_dev,
                            const double *S_dev, double *F_dev, void *cuda_stream);

/* Periodic systems (Eq. HamPeriodic, Eq. RealSpaceHamPeriodic, Eq. Bloch-basis). The real-space
 * matrix h^uc over the N_rs functions that can be non-zero in the unit cell is integrated by the
 * same code as a finite system: a handle whose atoms are the periodic images of the cell's atoms
 * and whose points are the unit cell's points (nao_integrate_h gives h^uc, NAO_TERM_POTENTIAL with
 * v = 1 gives s^uc).
 * nao_periodic_images (host): the images R_A + n1 a1 + n2 a2 + n3 a3 of the atoms atom_xyz
 * [n_atoms*3] whose fractional coordinates lie within `reach` (bohr; the largest cutoff radius)
 * of the cell [0, 1)^3 along every lattice direction (a superset of the images whose functions
 * reach the cell; the handle's relevance step drops the rest), the atoms themselves (n = 0) first.
 * lattice: host [9], rows a1, a2, a3. Outputs (host, caller-allocated, max_images entries):
 * img_xyz [3*n], img_atom [n] (the unit-cell atom), img_cell [3*n] (n1, n2, n3); *n_images = n.
 * n > max_images: NAO_ERR_INVALID_ARG with *n_images set (call again with room).
 * nao_periodic_basis_map (host): for the image system's basis (image atom -> radial function -> m),
 * fn_map[r] = the unit-cell basis index and fn_image[r] = the image of each of its N_rs functions;
 * *n_rs = N_rs (> max_rs: NAO_ERR_INVALID_ARG with *n_rs set).
 * nao_bloch_sum (GPU): hk_dev[2*((q*nb + i)*nb + j) + {0, 1}] = (re, im) of
 *     h_ij(k_q) = sum_{r -> i, s -> j} h_uc[r*n_rs + s] e^{i k_q . (T_s - T_r)},  T = img_cell A,
 * for the n_k points k_dev [n_k*3] (cartesian, 1/bohr): Eq. Bloch-basis inserted into
 * Eq. HamPeriodic. h_uc_dev [n_rs*n_rs], fn_map_dev/fn_image_dev [n_rs], img_cell_dev [3*n_images]
 * on the device; lattice on the host; hk_dev overwritten. FP64 atomics (one per element and k).
 * Every fn_map entry must lie in [0, nb) and every fn_image entry in [0, n_images), as
 * nao_periodic_basis_map writes them; the maps live on the device, so the kernel checks them
 * itself: an h^uc element with an out-of-range entry is skipped (nothing outside hk_dev and
 * img_cell_dev is touched) and counted into *err_dev, a device int32 the call zeroes first
 * (err_dev may be NULL: no count). Errors: NAO_ERR_INVALID_ARG, NAO_ERR_CUDA.                     */
nao_status nao_periodic_images(const double *atom_xyz, int32_t n_atoms, const double *lattice, double reach,
                               int32_t max_images, double *img_xyz, int32_t *img_atom, int32_t *img_cell,
                               int32_t *n_images);
nao_status nao_periodic_basis_map(const int32_t *atom_species, int32_t n_atoms, const int32_t *species_fn_offset,
                                  int32_t n_species, const int32_t *fn_l, const int32_t *img_atom, int32_t n_images,
                                  int64_t max_rs, int32_t *fn_map, int32_t *fn_image, int64_t *n_rs);
nao_status nao_bloch_sum(const double *h_uc_dev, int64_t n_rs, const int32_t *fn_map_dev, const int32_t *fn_image_dev,
                         const int32_t *img_cell_dev, int32_t n_images, const double *lattice, const double *k_dev,
                         int32_t n_k, int64_t nb, double *hk_dev, int32_t *err_dev, void *cuda_stream);

/* The same two operations with HOST buffers: the library copies the inputs to the device,
 * runs the operation on the given stream, copies the results back and synchronises the
 * stream before returning. Host buffers may be pageable or pinned (pinned is faster).
 * v_host may be NULL (v = 1); n_electrons_host may be NULL.                                */
nao_status nao_integrate_h_host(nao_grid *g, const double *v_host, uint32_t terms, nao_precision prec,
                                double *H_host, void *cuda_stream);
nao_status nao_update_density_host(nao_grid *g, const double *P_host, nao_precision prec, double *n_host,
                                   double *n_electrons_host, void *cuda_stream);

/* Basis functions of one batch (Sec. 3.4, the evaluation phase), for parity checks:
 * phi_dev[j*P_b + q] = phi_{rel_j}(r_q) and grad_dev[(c*N_b + j)*P_b + q] = d/dx_c of it,
 * for the batch's q = 0..P_b-1 points in batch order and j = 0..N_b-1 reduced-basis
 * positions. grad_dev may be NULL; for a batch with N_b = 0 nothing is written and both
 * pointers may be NULL. prec selects the evaluation arithmetic
 * (NAO_FP32 evaluates in FP32 and widens; NAO_FP64 and NAO_SPLIT evaluate in FP64).      */
nao_status nao_evaluate_batch(nao_grid *g, int64_t batch, nao_precision prec, double *phi_dev, double *grad_dev,
                              void *cuda_stream);

/* Kernel timing. When enabled, every kernel launch the handle makes is bracketed by CUDA
 * events recorded on the call's stream; nao_profile_read synchronises the device, converts
 * the event pairs to milliseconds and returns per kernel family the number of launches and
 * their summed duration (optionally resetting the record). Families are indexed by
 * nao_kernel_id.                                                                         */
typedef enum {
    NAO_K_EVAL_GRAD = 0, /* phi and grad phi of a chunk of batches */
    NAO_K_EVAL_PHI,      /* phi alone (density)                    */
    NAO_K_H_FP64,        /* FP64 h[B] contraction + scatter into H */
    NAO_K_H_FP32,        /* FP32 h[B] contraction + scatter        */
    NAO_K_H_SPLIT,       /* tensor-core slice products + scatter   */
    NAO_K_SLICE,         /* Ozaki slicing for H (weighted phi, grad phi) */
    NAO_K_MIRROR,        /* upper -> lower triangle copy of H      */
    NAO_K_N_FP64,        /* FP64 density contraction               */
    NAO_K_N_FP32,        /* FP32 density contraction               */
    NAO_K_N_SPLIT,       /* tensor-core density contraction        */
    NAO_K_REDUCE,        /* electron-count reduction               */
    NAO_K_SLICE_N,       /* Ozaki slicing for the density (phi, P') */
    NAO_K_COUNT
} nao_kernel_id;

typedef struct {
    int64_t launches[NAO_K_COUNT];
    double ms[NAO_K_COUNT];
} nao_profile;

nao_status nao_profile_enable(nao_grid *g, int32_t enable);
nao_status nao_profile_read(nao_grid *g, nao_profile *out, int32_t reset);

/* Hamiltonian integration that allocates nothing. The paper has no counterpart; this is a
 * library convenience. Some callers cannot allocate device memory where they integrate:
 * an application whose own memory manager owns all device memory, or a latency-bound loop
 * that must not call cudaMalloc/cudaFree (they can synchronise the device). This call
 * computes the same H as nao_integrate_h with NAO_FP64 (same kernels) but evaluates the
 * basis functions into a fixed device array of NAO_NOALLOC_SCRATCH_BYTES compiled into the
 * library, and calls no allocating routine.
 *   - The handle's evaluation chunks must fit the array: create the handle with
 *     options.scratch_bytes <= NAO_NOALLOC_SCRATCH_BYTES; otherwise NAO_ERR_INVALID_ARG and
 *     nothing is enqueued.
 *   - Every GPU that loads the library holds the array until the process exits.
 *   - All calls on a device share the array; it keeps the last call's contents (nothing in
 *     it needs clearing: every entry read is first written by the same call). Calls whose
 *     work overlaps on the GPU (other streams or handles) race on it.
 *   - The first call on a device looks up the array's device address; make that first call
 *     before any stream capture. The address is kept for the rest of the process: after a
 *     cudaDeviceReset (or any teardown of the device's primary context) the library's module
 *     is loaded again and the array may move, so this entry point must not be used on that
 *     device again in the same process.
 * Arguments and errors as nao_integrate_h (no precision argument: FP64).                    */
#define NAO_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
nao_status nao_integrate_h_noalloc(nao_grid *g, const double *v_dev, uint32_t terms, double *H_dev,
                                   void *cuda_stream);

/* Wait for the handle's enqueued work and report a device-side failure, if any: a bounded
 * device wait that gave up (NAO_ERR_TIMEOUT; its kernel skipped the rest of its work, so that
 * call's results are incomplete). The failure is reported once: the handle's error word is
 * cleared, and later calls run normally.                                                    */
nao_status nao_sync_status(nao_grid *g);

/* Failure handling without a GPU fault (the paper has no counterpart; test support).
 * nao_fault_inject: makes the n-th device allocation ("alloc:<n>"), host<->device copy
 * ("copy:<n>") or kernel launch ("launch:<n>") that the library attempts after this call fail
 * once, as if the CUDA call had failed (nothing is allocated, copied or launched for it). The
 * entry point that hits it returns NAO_ERR_OUT_OF_MEMORY (allocation) or NAO_ERR_CUDA with a
 * message that starts "injected failure"; a create leaves *out NULL, a call on a handle leaves the
 * handle usable and destroyable (its outputs of that call are undefined). Process-wide; NULL or ""
 * clears a pending injection; the environment variable NAO_FAULT_INJECT sets the same the first
 * time the library needs it. Errors: NAO_ERR_INVALID_ARG (malformed spec).
 * nao_check_wait_timeout: enqueues one bounded device wait (the mbarrier wait of the tensor-core
 * pipelines) on a barrier that nothing completes; after max_cycles SM cycles (1..2^34) it gives
 * up and records NAO_ERR_TIMEOUT in the handle's error word, as a stuck pipeline would, for
 * nao_sync_status to report. Nothing else is touched.                                          */
nao_status nao_fault_inject(const char *spec);
nao_status nao_check_wait_timeout(nao_grid *g, int64_t max_cycles, void *cuda_stream);

/* Static text for a status code. */
const char *nao_status_string(nao_status s);

/* Text of the most recent failure on the calling thread (empty if none). */
const char *nao_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NAO_H */

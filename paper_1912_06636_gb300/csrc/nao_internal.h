// Internal declarations of libnao: the handle, kernel argument blocks and launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>
#include <map>
#include <vector>

#include "nao.h"

#define NAO_LMAX 6
#define NAO_TILE 64          // tile edge of the SIMT contractions (basis functions and points)
#define NAO_PPAD 16          // batch points are padded to a multiple of this in scratch
#define NAO_MAX_BATCH 1024   // largest accepted max_batch_points
#define NAO_SPLIT_MAX_SLICES 12  // bf16 digits: S groups x TN FP32 columns <= 512 tensor-memory columns
#define NAO_SPLIT_MAX_SLICES_E4M3 16  // e4m3 digits (TN = 32): 16 x 32 = 512 columns
#define NAO_SPLIT_MAX_PPAD 512   // split path: padded batch points (the slicers' shared-memory column tables)

// One radial function instance relevant to a batch: atom, radial function, position of
// its m = -l entry in the batch's reduced basis, l.
struct RfnEntry {
    int32_t atom, fn, pos, l;
};

// The relevant radial functions of one atom for one batch: rfn entries [r0, r0 + nr), sorted
// by l; lmax is the largest l among them.
struct AtomGroup {
    int32_t atom, r0, nr, lmax;
};

// Systems of a handle. A handle holds one or more systems (molecules); batches never mix
// systems and every basis index, atom and point is global (systems concatenated). The
// per-call pointer tables (H, v, P, n, N_e) are device arrays with one entry per system,
// written before each call's kernels.
struct SysTables {
    const int32_t *bmol;     // [n_batches] system of each batch
    const int32_t *boff;     // [n_sys] first global basis index of the system
    const int32_t *nbm;      // [n_sys] basis size of the system
    const int32_t *poff;     // [n_sys] first global point (caller's order) of the system
    const int32_t *aoff;     // [n_sys + 1] atoms of the system
    double *const *H;        // [n_sys] this call's H of each system (nbm x nbm)
    const double *const *v;  // [n_sys] this call's v of each system (NULL entry: v = 1)
    const double *const *P;  // [n_sys] this call's P of each system
    double *const *n;        // [n_sys] this call's n of each system
    double *const *ne;       // [n_sys] this call's N_e of each system (NULL entry: not formed)
    double *const *gn;       // [n_sys] this call's grad n of each system ([3][np], component-major)
    const double *const *vt; // [n_sys] this call's v_tau of each system (NULL entry: no tau term)
    unsigned long long *const *Hacc;  // [n_sys] deterministic mode: the system's H as 128-bit fixed-point
                                      // integers (lo, hi per element); NULL entries: FP64 atomics into H
    const int32_t *np;       // [n_sys] points of the system
};

// Geometry and tables shared by every kernel (device pointers).
struct DevSystem {
    const double *atom_xyz;   // [n_atoms*3]
    const double *coef;       // [n_fn][n_rgrid-1][4] spline coefficients in t
    const float *coef_f32;    // same in FP32 (rounded to nearest)
    const float *coef_lo;     // c - coef_f32 rounded to FP32: (coef_f32, coef_lo) is c as a float-float
    const double *inv_rk;     // [n_rgrid] 1 / r_k of the logarithmic grid
    const uint8_t *seg64;     // [n_fn][n_rgrid-1] 1: the FP32 path evaluates this spline segment in FP64
    const double *fn_rc;      // [n_fn]
    const double *px, *py, *pz, *pw;  // points in batch order
    const int32_t *perm;      // batch order -> original index
    const int32_t *batch_off; // [n_batches+1]
    const int32_t *rel_off;   // [n_batches+1]
    const int32_t *rel_idx;   // [rel_total]
    const int32_t *rfn_off;   // [n_batches+1]
    const RfnEntry *rfn;      // [rfn_total]
    const int32_t *agrp_off;  // [n_batches+1] atom groups of each batch
    const AtomGroup *agrp;    // [agrp_total]
    const int64_t *scr_off;   // [n_batches] element offset of the batch's block in scratch
    int32_t n_rgrid;
    double r0, inv_delta;
    double step_m1;           // exp(Delta) - 1: r_{k+1} / r_k - 1 of the logarithmic grid
    int64_t nb;               // total basis size over all systems
    SysTables sys;
    double knorm[NAO_LMAX + 1][NAO_LMAX + 1];  // sqrt((2l+1)/(4pi) (l-m)!/(l+m)!) (x sqrt2 for m>0)
    float knorm_h[NAO_LMAX + 1][NAO_LMAX + 1], knorm_l[NAO_LMAX + 1][NAO_LMAX + 1];  // knorm as float-float
};

#ifdef __CUDACC__
// Element (i, j) of the H of system m (i, j global basis indices of that system).
__device__ __forceinline__ double *h_elem(const DevSystem &s, int m, int64_t gi, int64_t gj) {
    const int64_t bo = s.sys.boff[m];
    return s.sys.H[m] + (gi - bo) * (int64_t)s.sys.nbm[m] + (gj - bo);
}

// Deterministic accumulation: x is added as the 128-bit two's-complement integer X = round(x 2^90)
// (|x| < 2^37), low word first; a wrap of the unsigned low word carries one into the high word.
// Integer addition is associative, so the final (hi, lo) of an element, and the FP64 value the
// mirror pass makes of it, do not depend on the order of the additions.
constexpr int NAO_DET_FRAC = 90;
__device__ __forceinline__ void det_add(unsigned long long *acc, double x) {
    const double y = x * 0x1p26;  // x 2^(90 - 64), exact
    const double f = floor(y);
    long long hi = (long long)f;
    const double fr = rint((y - f) * 0x1p64);  // the fraction in units of 2^-90: [0, 2^64]
    unsigned long long lo;
    if (fr >= 0x1p64) {
        lo = 0ULL;
        hi += 1;
    } else {
        lo = (unsigned long long)fr;
    }
    const unsigned long long old = atomicAdd(acc, lo);
    atomicAdd(acc + 1, (unsigned long long)hi + (old + lo < old ? 1ULL : 0ULL));
}
__device__ __forceinline__ double det_value(const unsigned long long *acc) {
    return fma((double)(long long)acc[1], 0x1p-26, (double)acc[0] * 0x1p-90);
}

// H_ij += x for system m: an FP64 atomic, or the deterministic fixed-point addition.
__device__ __forceinline__ void h_add(const DevSystem &s, int m, int64_t gi, int64_t gj, double x) {
    unsigned long long *acc = s.sys.Hacc[m];
    if (acc) {
        const int64_t bo = s.sys.boff[m];
        det_add(acc + 2 * ((gi - bo) * (int64_t)s.sys.nbm[m] + (gj - bo)), x);
    } else {
        atomicAdd(h_elem(s, m, gi, gj), x);
    }
}
__device__ __forceinline__ double p_elem(const DevSystem &s, int m, int64_t gi, int64_t gj) {
    const int64_t bo = s.sys.boff[m];
    return s.sys.P[m][(gi - bo) * (int64_t)s.sys.nbm[m] + (gj - bo)];
}
// v at batch-ordered point p of system m (1 when the system has no v this call).
__device__ __forceinline__ double v_at(const DevSystem &s, int m, int p) {
    const double *v = s.sys.v[m];
    return v ? v[s.perm[p] - s.sys.poff[m]] : 1.0;
}
// v_tau at batch-ordered point p of system m (0 when the system has no v_tau this call).
__device__ __forceinline__ double vt_at(const DevSystem &s, int m, int p) {
    const double *vt = s.sys.vt[m];
    return vt ? vt[s.perm[p] - s.sys.poff[m]] : 0.0;
}
__device__ __forceinline__ double *n_at(const DevSystem &s, int m, int p) {
    return s.sys.n[m] + (s.perm[p] - s.sys.poff[m]);
}
// component c of grad n at batch-ordered point p of system m
__device__ __forceinline__ double *gn_at(const DevSystem &s, int m, int p, int c) {
    return s.sys.gn[m] + (int64_t)c * s.sys.np[m] + (s.perm[p] - s.sys.poff[m]);
}
#endif

// Digit formats of the split path (options.split_digits):
//   NAO_DIGITS_BF16: balanced base-64 digits, |d| <= 32, stored as bf16, tcgen05 kind::f16 MMAs
//                    with K = 16 per instruction;
//   NAO_DIGITS_E4M3: balanced base-32 digits, |d| <= 16 (every such integer is exact in e4m3),
//                    stored as e4m3 bytes, kind::f8f6f4 MMAs with K = 32 at twice the bf16 rate.
// Either way a 128-byte operand row holds one K chunk (64 bf16 or 128 e4m3 columns) and an MMA
// K step is 32 bytes, so the shared-memory descriptors, the 128-byte swizzle and the four K
// steps per chunk are the same; a digit product is at most 2^(2 bits - 2) (2^10 or 2^8).
#define NAO_DIGITS_BF16 0
#define NAO_DIGITS_E4M3 1
__host__ __device__ constexpr int nao_digit_bits(int F) { return F == NAO_DIGITS_E4M3 ? 5 : 6; }
__host__ __device__ constexpr int nao_chunk_cols(int F) { return F == NAO_DIGITS_E4M3 ? 128 : 64; }
__host__ __device__ constexpr int nao_kstep_cols(int F) { return F == NAO_DIGITS_E4M3 ? 32 : 16; }
// Largest K of one exact accumulation of S slice groups: K S 2^(2 bits - 2) < 2^24.
__host__ __device__ constexpr int nao_exact_ks(int F) { return F == NAO_DIGITS_E4M3 ? 65536 : 16384; }

// Geometry of one batch's operand slices on the split path (shared by host and device code).
// Every operand is stored row-contiguous per (slice, K chunk): rows x 128 B with the 128-byte
// swizzle inside 8-row atoms, rows rounded up to 16 only. An MMA tile (128 rows for A, TN for B)
// is a plain byte range; the last tile of an operand is copied short and its remaining
// shared-memory rows keep stale data, which only reaches output rows and columns beyond N (or P)
// that the epilogues discard. B tiles are TN = nao_split_tn(S, F) rows.
// H: one digit set, rows = basis functions, K = the 4 Ppad weighted columns reordered so that
//    negative-weight columns come first, padded to a whole MMA K step (B negated on those steps).
// Density: A rows = points, K = basis; B rows = basis (P' rows), K = basis.
// MMA N (rows of a B tile) of the split path with S slices: each of the S slice groups holds
// its own TN FP32 accumulator columns of the 512 tensor-memory columns.
__host__ __device__ constexpr int nao_split_tn(int S, int F = NAO_DIGITS_BF16) {
    return F == NAO_DIGITS_BF16 && S <= 10 ? 48 : 32;
}

struct SplitGeom {
    int n_kc, R16;               // H: K chunks, stored rows
    int n_kcN, P16, n_qt, n_jtN; // density: K chunks, stored A rows, 128-point tiles, TN-row B tiles
    __host__ __device__ SplitGeom(int P, int N, int S, int TN = 0, int F = NAO_DIGITS_BF16) {
        if (TN == 0) TN = nao_split_tn(S, F);
        const int C = nao_chunk_cols(F), ks = nao_kstep_cols(F);
        const int Ppad = (P + NAO_PPAD - 1) / NAO_PPAD * NAO_PPAD;
        n_kc = (4 * Ppad + ks + C - 1) / C;
        R16 = (N + 15) / 16 * 16;
        n_kcN = (N + C - 1) / C;
        P16 = (P + 15) / 16 * 16;
        n_qt = (P + 127) / 128;
        n_jtN = (N + TN - 1) / TN;
    }
    __host__ __device__ size_t h_block(int s, int kc) const { return ((size_t)s * n_kc + kc) * (size_t)R16 * 128; }
    __host__ __device__ size_t h_bytes(int S) const { return (size_t)S * n_kc * (size_t)R16 * 128; }
    __host__ __device__ int h_slice_tiles() const { return (R16 + 63) / 64; }
    __host__ __device__ size_t nA_block(int s, int kc) const { return ((size_t)s * n_kcN + kc) * (size_t)P16 * 128; }
    __host__ __device__ size_t n_setA(int S) const { return (size_t)S * n_kcN * (size_t)P16 * 128; }
    __host__ __device__ size_t nB_block(int S, int s, int kc) const {
        return n_setA(S) + ((size_t)s * n_kcN + kc) * (size_t)R16 * 128;
    }
    __host__ __device__ size_t n_bytes(int S) const { return n_setA(S) + (size_t)S * n_kcN * (size_t)R16 * 128; }
};

struct HWork {  // one upper-triangular tile pair of one batch's h[B] (Eq. batch_matrix_mult)
    int32_t batch, ti, tj, pad;  // split H items: pad = the K segment (below)
};

// K segments of the split H contraction. A slice-order group's FP32 accumulator sums K products
// of at most 2^(2 bits - 2) for each of its g + 1 <= S slice pairs; it stays an exact integer
// while K S 2^(2 bits - 2) < 2^24 (nao_exact_ks). A batch whose 4 Ppad weighted columns meet that
// bound is one accumulation; a larger batch is accumulated in segments of nao_split_kc_seg(S, F)
// K chunks, each recombined and scattered into H on its own (H is a sum over K, so the segments'
// FP64 partial sums simply add; Eq. H_decomp).
__host__ __device__ constexpr int nao_split_kc_seg(int S, int F = NAO_DIGITS_BF16) {
    return (nao_exact_ks(F) - 1) / (nao_chunk_cols(F) * S);
}
__host__ __device__ inline int nao_split_h_nseg(int P, int S, int F = NAO_DIGITS_BF16) {
    const int Ppad = (P + NAO_PPAD - 1) / NAO_PPAD * NAO_PPAD;
    if (4 * Ppad * S < nao_exact_ks(F)) return 1;
    const int C = nao_chunk_cols(F);
    const int n_kc = (4 * Ppad + nao_kstep_cols(F) + C - 1) / C, kcs = nao_split_kc_seg(S, F);
    return (n_kc + kcs - 1) / kcs;
}
// K chunks [kc0, kc1) of segment seg of a batch with n_kc chunks.
__host__ __device__ inline void nao_split_h_seg_range(int n_kc, int nseg, int seg, int S, int &kc0, int &kc1,
                                                      int F = NAO_DIGITS_BF16) {
    if (nseg <= 1) {
        kc0 = 0;
        kc1 = n_kc;
        return;
    }
    const int kcs = nao_split_kc_seg(S, F);
    kc0 = seg * kcs;
    kc1 = kc0 + kcs < n_kc ? kc0 + kcs : n_kc;
}

// Split H work items of one batch (P points, N functions) for tile width TN and S slices: per
// 128-row tile I, the TN-column tiles J >= floor(128 I / TN) (those reaching the upper
// triangle), once per K segment.
inline void nao_split_h_items(int32_t b, int P, int N, int TN, int S, std::vector<HWork> &out,
                              int F = NAO_DIGITS_BF16) {
    const int nI = (N + 127) / 128, nJ = (N + TN - 1) / TN, nseg = nao_split_h_nseg(P, S, F);
    for (int I = 0; I < nI; I++)
        for (int J = (I * 128) / TN; J < nJ; J++)
            for (int q = 0; q < nseg; q++) out.push_back({b, I, J, q});
}
struct DWork {  // one tile of points of one batch for the density
    int32_t batch, tp;
};

struct Chunk {  // a run of batches whose evaluated basis functions fit the scratch at once
    int32_t b0, b1;
    int32_t hw0, hw1;  // H work items of these batches
    int32_t dw0, dw1;  // density work items of these batches
};

struct nao_grid {
    int device = 0;
    nao_options opt{};
    // host copies of the problem
    int32_t n_atoms = 0, n_species = 0, n_fn = 0, n_rgrid = 0;
    int64_t nb = 0, n_points = 0, n_batches = 0, rel_total = 0, rfn_total = 0;
    double r0 = 0, r_last = 0, delta = 0;
    std::vector<int64_t> batch_off, perm, rel_off;
    std::vector<int32_t> rel_idx;
    std::vector<int32_t> Pb, Nb;
    int32_t max_P = 0, max_N = 0;
    int64_t flops_h = 0, flops_n = 0;
    std::vector<Chunk> chunks;
    int64_t scratch_elems = 0;  // doubles
    int64_t n_hwork = 0, n_dwork = 0;
    // device memory: stream-ordered allocations from the library's per-device pool, made and
    // freed on the handle's own setup stream (no device-wide synchronisation at create or
    // destroy); ev_last marks the end of the handle's most recently enqueued call
    std::vector<void *> allocs;
    int64_t dev_bytes = 0;
    cudaStream_t setup = nullptr;
    cudaEvent_t ev_last = nullptr;
    bool used = false, counted = false;
    DevSystem sys{};
    HWork *d_hwork = nullptr;
    DWork *d_dwork = nullptr;
    double *d_scratch = nullptr;
    double *d_ne_part = nullptr;    // [n_dwork] per-tile sums of w n
    int32_t *d_err = nullptr;       // device error word
    // systems (molecules) of the handle
    int32_t n_sys = 1;
    std::vector<int32_t> sys_boff, sys_nb, sys_poff, sys_np, sys_aoff;
    std::vector<int32_t> sys_dw0;      // [n_sys + 1] density work items of each system
    std::vector<int4> zero_tasks;      // (system, start element, count, 0) chunks of each H
    std::vector<int4> mirror_tasks;    // (system, column tile, row tile, 0) with row <= column
    int4 *d_zero_tasks = nullptr, *d_mirror_tasks = nullptr;
    int32_t *d_sys_dw0 = nullptr, *d_sys_np = nullptr;
    double **d_tab = nullptr;          // device: [6][n_sys] pointer tables H, v, P, n, N_e, grad n
    std::vector<void *> h_tab;         // host copy of the tables
    // split (tensor-core) path, set up on its first use
    struct SplitChunk {
        int32_t b0, b1;    // batches (inside one chunk of the evaluation scratch)
        int32_t max_rt, max_qt;  // grid extents of the slicing kernels
        // items of the split H and density lists: [0] tile width 48, [1] tile width 32
        int32_t hw0[2], hw1[2];
        int32_t nw0[2], nw1[2];
    };
    bool split_ready = false;
    int split_S = 0, split_F = 0;  // slices and digit format of the split set-up
    std::vector<SplitChunk> split_chunks;
    // density Hessian (FP64): chunks of batches whose 10-row evaluation fits the scratch, with
    // their density work ranges, and the per-batch scratch offsets of that layout
    struct HessChunk {
        int32_t b0, b1, dw0, dw1;
    };
    std::vector<HessChunk> hess_chunks;
    int64_t *d_hess_off = nullptr;
    // density Hessian on the split path: ranges of batches inside one Hessian chunk and one
    // split chunk, with their own density work items (rebuilt when the tile widths change)
    struct HessSplitSub {
        int32_t b0, b1, max_qt, max_rt;
        int32_t nw0[2], nw1[2];  // items of width 48, 32 in d_hess_nw
    };
    std::vector<HessSplitSub> hess_split;
    HWork *d_hess_nw = nullptr;
    int64_t cap_hess_nw = 0;
    int32_t *d_expo4 = nullptr;  // [4][n_points] point exponents of phi, d/dx, d/dy, d/dz phi
    int split_lists_ver = 0, hess_split_ver = -1;
    // local Pulay force terms: every 64 x 64 tile pair of every batch, per Hessian chunk
    std::vector<int64_t> atom_basis;         // [n_atoms + 1] first global basis index of each atom
    std::vector<int32_t> pulay_w0;           // [hess_chunks + 1] work ranges
    HWork *d_pulay_work = nullptr;
    int64_t *d_atom_basis = nullptr;
    // tile width (MMA N) of every batch on the split path: a fixed rule until the autotuner has
    // timed both widths per (N_b, P_b) bucket of the batch-size histogram
    std::vector<int32_t> split_tn;
    int32_t *d_split_tn = nullptr;
    bool split_tuned = false;
    int32_t tune_buckets = 0;      // buckets the autotuner timed
    int64_t cap_split_hw = 0, cap_split_nw = 0;
    HWork *d_tune_hw = nullptr;    // scratch work list of the autotuner
    int64_t cap_tune_hw = 0;
    uint8_t *d_slices = nullptr;
    int64_t *d_sl_off_h = nullptr, *d_sl_off_n = nullptr;
    int32_t *d_expo_h = nullptr, *d_expo_q = nullptr, *d_expo_b = nullptr;
    int32_t *d_neg16 = nullptr;  // per batch: leading negative-weight K steps of 16 columns
    HWork *d_split_hw = nullptr, *d_split_nw = nullptr;
    int64_t n_split_hw = 0, n_split_nw = 0;
    // kernel timing (nao_profile_enable)
    bool profiling = false;
    struct Timed {
        int kid;
        cudaEvent_t a, b;
    };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
    nao_profile prof{};
    // staging for the host-buffer entry points (allocated on first use)
    double *d_stage_in = nullptr, *d_stage_out = nullptr, *d_stage_ne = nullptr;
    // CUDA graphs (options.capture_graph): one executable graph per (operation, precision,
    // terms), replayed on the handle's own stream between two events
    cudaStream_t gstream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::map<uint64_t, cudaGraphExec_t> graphs;
};

// ---- launchers (eval.cu, contract_simt.cu) ----------------------------------------------
// minr2[b * max_atoms + a]: min over batch b's points of |r - R_A|^2 for the a-th atom of b's
// system (atoms aoff[m] .. aoff[m+1]-1).
cudaError_t launch_relevance_minr2(const double *atom_xyz, const int32_t *bmol, const int32_t *aoff, int32_t max_atoms,
                                   const double *px, const double *py, const double *pz, const int32_t *batch_off,
                                   int64_t n_batches, double *minr2, cudaStream_t st);
cudaError_t launch_eval(const DevSystem &s, int32_t b0, int32_t b1, nao_precision prec, bool grad, double *scratch,
                        cudaStream_t st);
// Split path, the density's evaluation (FP64 values; phi, with grad phi when grad) and the
// point exponents of the slicing into expo (by batch-ordered point; n_red >= P_b).
cudaError_t launch_eval_split(const DevSystem &s, int32_t b0, int32_t b1, bool grad, double *scratch, int32_t *expo,
                              int32_t n_red, cudaStream_t st);
// Density Hessian (FP64, or FP32 with fp32): evaluation of phi, grad phi and the six second
// derivatives (computed in FP64, stored as double or float: 10 rows of Ppad per function at
// scratch + hoff[b] elements; lap: the fifth row holds the Laplacian, for the Pulay terms) and
// the contraction in the same type (n, grad n into the pointer
// tables' sections 3 and 5, the Hessian component-major into hess, per-tile w n into ne_part).
cudaError_t launch_eval_hess(const DevSystem &s, int32_t b0, int32_t b1, void *scratch, bool fp32, bool lap,
                             const int64_t *hoff, cudaStream_t st);
cudaError_t launch_density_hess(const DevSystem &s, const DWork *work, int32_t w0, int32_t n_work, const void *scratch,
                                bool fp32, const int64_t *hoff, double *hess, double *ne_part, cudaStream_t st);
// Local Pulay force terms (FP64, or FP32 with fp32, from the Hessian evaluation of the same
// type): M^c += sum_q w d_c phi_i (-1/2 lap + v) phi_j and S^c += sum_q w d_c phi_i phi_j over the
// full tile pairs of work items (batch, I, J), into M and S ([3][nb][nb], single system); and
// F[3 a + c] = 2 sum_{i on a} sum_j (n_ij M^c_ij - q_ij S^c_ij).
cudaError_t launch_pulay(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const void *scratch, bool fp32,
                         const int64_t *hoff, double *M, double *S, int64_t nb, cudaStream_t st);
cudaError_t launch_pulay_forces(const double *nmat, const double *qmat, const double *M, const double *S,
                                const int64_t *atom_basis, int32_t n_atoms, int64_t nb, double *F, cudaStream_t st);
cudaError_t launch_eval_one(const DevSystem &s, int32_t b, nao_precision prec, double *phi, double *grad,
                            cudaStream_t st);
cudaError_t launch_h_simt(const DevSystem &s, nao_precision prec, const HWork *work, int32_t n_work,
                          const double *scratch, uint32_t terms, cudaStream_t st);
cudaError_t launch_zero_h(const DevSystem &s, const int4 *tasks, int32_t n_tasks, cudaStream_t st);
cudaError_t launch_mirror(const DevSystem &s, const int4 *tasks, int32_t n_tasks, cudaStream_t st);
// grad: also grad n = 2 sum_j T_qj grad phi_jq with T = Phi P over all of P (the scratch then holds
// phi and grad phi, rows of 4 Ppad)
cudaError_t launch_density_simt(const DevSystem &s, nao_precision prec, const DWork *work, int32_t w0, int32_t n_work,
                                const double *scratch, double *ne_part, bool grad, cudaStream_t st);
// N_e of every system: sum of its density work items' partial sums (deterministic order)
cudaError_t launch_reduce_ne(const DevSystem &s, const double *part, const int32_t *sys_dw0, int32_t n_sys,
                             cudaStream_t st);
// dst[i] = src[i] for i < n, written by kernels whose arguments carry the pointer values (no host
// buffer has to outlive the call)
cudaError_t launch_set_pointers(double **dst, void *const *src, int32_t n, cudaStream_t st);
// n = 0 at every point of the given density work items
cudaError_t launch_zero_n(const DevSystem &s, const DWork *work, int32_t n_work, bool grad, cudaStream_t st);

// ---- split path (split_tc.cu) ------------------------------------------------------------
// F: digit format (NAO_DIGITS_BF16, NAO_DIGITS_E4M3) in every split launcher below
size_t split_smem_bytes(int S, int F);
cudaError_t split_configure();
cudaError_t launch_slice_h(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_rt, const double *scratch,
                           uint32_t terms, uint8_t *slices, const int64_t *sl_off, int32_t *expo, int32_t *neg16, int S,
                           int F, cudaStream_t st);
// tn: tile width 48 (bf16 digits, S <= 10 only) or 32; scatter = 0 skips the H scatter (autotuner timing).
// work: items (batch, 128-row tile I, TN-column tile J) of nao_split_h_items; a persistent kernel
// (one CTA per SM) walks them
cudaError_t launch_h_tc(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                        const int64_t *sl_off, const int32_t *expo, const int32_t *neg16, int S, int F, int tn,
                        int scatter, int32_t *err, cudaStream_t st);
// tn_b: per-batch tile width (the P' tiles of the density follow it). grad: the scratch rows hold
// [phi | grad phi] (4 Ppad) and P' = P over all tiles (density gradient)
cudaError_t launch_slice_n(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_qt, int32_t max_rt,
                           const double *scratch, uint8_t *slices, const int64_t *sl_off, const int32_t *expo_q,
                           int32_t *expo_b, const int32_t *tn_b, int S, int F, bool grad, cudaStream_t st);
// The density Hessian on the split path (passes comp = 0..3 over the 10-row FP64 evaluation at
// hoff: A = phi, then the gradient components; P' sliced with the first pass): slicing, the
// four A operands' point exponents (expo4[comp n_points + p]) and the contraction passes
// (comp 0 writes n, grad n and hess; comp a adds hess_(a, b), b >= a).
cudaError_t launch_slice_n_hess(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_qt, int32_t max_rt,
                                const double *scratch, const int64_t *hoff, int comp, uint8_t *slices,
                                const int64_t *sl_off, const int32_t *expo_q, int32_t *expo_b, const int32_t *tn_b, int S,
                                int F, cudaStream_t st);
cudaError_t launch_hess_point_expo(const DevSystem &s, int32_t b0, int32_t b1, const double *scratch, const int64_t *hoff,
                                   int32_t *expo4, int64_t n_points, cudaStream_t st);
cudaError_t launch_n_tc_hess(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                             const int64_t *sl_off, const int32_t *expo_q, const int32_t *expo_b, const double *scratch,
                             const int64_t *hoff, int comp, double *hess, int S, int F, int tn, int32_t *err,
                             cudaStream_t st);
cudaError_t launch_n_tc(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                        const int64_t *sl_off, const int32_t *expo_q, const int32_t *expo_b, const double *scratch, int S,
                        int F, int tn, bool grad, int32_t *err, cudaStream_t st);
// One bounded mbarrier wait that nothing completes (the wait of the tensor-core pipelines): it gives
// up after max_cycles SM cycles and records NAO_ERR_TIMEOUT in err[0] (code 1 in err[1]).
cudaError_t launch_wait_timeout_probe(long long max_cycles, int32_t *err, cudaStream_t st);
cudaError_t launch_wn_partial(const DevSystem &s, const DWork *work, int32_t w0, int32_t n_work, double *ne_part,
                              cudaStream_t st);

// Records the text nao_last_error() returns on the calling thread (api.cpp).
void nao_set_last_error(const std::string &msg);

// ---- host helpers (partition.cpp) --------------------------------------------------------
// Recursive bisection (see nao_grid_create in nao.h); returns the number of batches.
int64_t nao_partition(int64_t n, const double *xyz, int64_t B, std::vector<int64_t> &offsets,
                      std::vector<int64_t> &perm);
// Natural cubic spline in the index coordinate: coefficients of y_k + c1 t + c2 t^2 + c3 t^3.
void nao_spline_coefficients(const double *y, int32_t n, double *coef /* [(n-1)*4] */);

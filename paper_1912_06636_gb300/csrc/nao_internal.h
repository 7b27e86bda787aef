// Internal declarations of libnao: the handle, kernel argument blocks and launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>
#include <vector>

#include "nao.h"

#define NAO_LMAX 6
#define NAO_TILE 64          // tile edge of the SIMT contractions (basis functions and points)
#define NAO_PPAD 16          // batch points are padded to a multiple of this in scratch
#define NAO_MAX_BATCH 1024   // largest accepted max_batch_points
#define NAO_SPLIT_MAX_SLICES 10  // tensor-memory budget: 10 groups x 48 FP32 columns <= 512 columns
#define NAO_SPLIT_TN 48          // split path: MMA N (B-tile rows)
#define NAO_SPLIT_MAX_PPAD 512   // split path: padded batch points (4 Ppad S < 2^14 keeps sums exact)

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

// Geometry and tables shared by every kernel (device pointers).
struct DevSystem {
    const double *atom_xyz;   // [n_atoms*3]
    const double *coef;       // [n_fn][n_rgrid-1][4] spline coefficients in t
    const float *coef_f32;    // same in FP32
    const double *inv_rk;     // [n_rgrid] 1 / r_k of the logarithmic grid
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
    int64_t nb;
    double knorm[NAO_LMAX + 1][NAO_LMAX + 1];  // sqrt((2l+1)/(4pi) (l-m)!/(l+m)!) (x sqrt2 for m>0)
};

// Geometry of one batch's operand slices on the split path (shared by host and device code).
// H: one digit set; per (slice, K chunk of 64) a row-contiguous block of R_pad rows x 128 B
//    (128-byte swizzle inside 8-row atoms), so a 128-row A tile and a 48-row B tile are plain
//    byte ranges. K holds the 4 Ppad weighted columns reordered so that negative-weight
//    columns come first, padded to a multiple of 16 (the MMA negates B on those K steps).
// Density: A rows (points) in 128-row blocks, K = basis in chunks of 64; B rows (basis) in
//    48-row blocks. One block = rows x 64 bf16, 128 B per row.
struct SplitGeom {
    int n_kc, R_pad;             // H: K chunks, padded rows
    int n_kcN, n_qt, n_jtN;      // density: K chunks, A 128-point blocks, B 48-row blocks
    __host__ __device__ SplitGeom(int P, int N) {
        const int Ppad = (P + NAO_PPAD - 1) / NAO_PPAD * NAO_PPAD;
        n_kc = (4 * Ppad + 16 + 63) / 64;
        const int ra = 128 * ((N + 127) / 128), rb = NAO_SPLIT_TN * ((N + NAO_SPLIT_TN - 1) / NAO_SPLIT_TN);
        R_pad = ra > rb ? ra : rb;
        n_kcN = (N + 63) / 64;
        n_qt = (P + 127) / 128;
        n_jtN = (N + NAO_SPLIT_TN - 1) / NAO_SPLIT_TN;
    }
    __host__ __device__ size_t h_block(int s, int kc) const { return ((size_t)s * n_kc + kc) * (size_t)R_pad * 128; }
    __host__ __device__ size_t h_bytes(int S) const { return (size_t)S * n_kc * (size_t)R_pad * 128; }
    __host__ __device__ int h_slice_tiles() const { return R_pad / 64 + (R_pad % 64 ? 1 : 0); }
    __host__ __device__ size_t n_setA(int S) const { return (size_t)S * n_kcN * n_qt * 16384; }
    __host__ __device__ size_t n_bytes(int S) const { return n_setA(S) + (size_t)S * n_kcN * n_jtN * (NAO_SPLIT_TN * 128); }
};

struct HWork {  // one upper-triangular tile pair of one batch's h[B] (Eq. batch_matrix_mult)
    int32_t batch, ti, tj, pad;
};
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
    // device memory
    std::vector<void *> allocs;
    int64_t dev_bytes = 0;
    DevSystem sys{};
    HWork *d_hwork = nullptr;
    DWork *d_dwork = nullptr;
    double *d_scratch = nullptr;
    double *d_ne_part = nullptr;    // [n_dwork] per-tile sums of w n
    int32_t *d_err = nullptr;       // device error word
    // split (tensor-core) path, set up on its first use
    struct SplitChunk {
        int32_t b0, b1;    // batches (inside one chunk of the evaluation scratch)
        int32_t hw0, hw1;  // items of the split H list
        int32_t nw0, nw1;  // items of the split density list
        int32_t max_rt, max_qt;  // grid extents of the slicing kernels
    };
    bool split_ready = false;
    int split_S = 0;
    std::vector<SplitChunk> split_chunks;
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
};

// ---- launchers (eval.cu, contract_simt.cu) ----------------------------------------------
cudaError_t launch_relevance_minr2(const double *atom_xyz, int32_t n_atoms, const double *px, const double *py,
                                   const double *pz, const int32_t *batch_off, int64_t n_batches, double *minr2,
                                   cudaStream_t st);
cudaError_t launch_eval(const DevSystem &s, int32_t b0, int32_t b1, nao_precision prec, bool grad, double *scratch,
                        cudaStream_t st);
cudaError_t launch_eval_one(const DevSystem &s, int32_t b, nao_precision prec, double *phi, double *grad,
                            cudaStream_t st);
cudaError_t launch_h_simt(const DevSystem &s, nao_precision prec, const HWork *work, int32_t n_work,
                          const double *scratch, const double *v, uint32_t terms, double *H, cudaStream_t st);
cudaError_t launch_mirror(double *H, int64_t nb, cudaStream_t st);
cudaError_t launch_density_simt(const DevSystem &s, nao_precision prec, const DWork *work, int32_t w0, int32_t n_work,
                                const double *scratch, const double *P, double *n, double *ne_part, cudaStream_t st);
cudaError_t launch_reduce_sum(const double *part, int64_t n, double *out, cudaStream_t st);

// ---- split path (split_tc.cu) ------------------------------------------------------------
size_t split_smem_bytes(int S);
cudaError_t split_configure();
cudaError_t launch_slice_h(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_rt, const double *scratch,
                           const double *v, uint32_t terms, uint8_t *slices, const int64_t *sl_off, int32_t *expo,
                           int32_t *neg16, int S, cudaStream_t st);
cudaError_t launch_h_tc(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                        const int64_t *sl_off, const int32_t *expo, const int32_t *neg16, int S, double *H, int32_t *err,
                        cudaStream_t st);
cudaError_t launch_slice_n(const DevSystem &s, int32_t b0, int32_t b1, int32_t max_qt, const double *scratch,
                           const double *P, uint8_t *slices, const int64_t *sl_off, int32_t *expo_q, int32_t *expo_b,
                           int S, cudaStream_t st);
cudaError_t launch_n_tc(const DevSystem &s, const HWork *work, int32_t w0, int32_t n_work, const uint8_t *slices,
                        const int64_t *sl_off, const int32_t *expo_q, const int32_t *expo_b, const double *scratch, int S,
                        double *n, int32_t *err, cudaStream_t st);
cudaError_t launch_wn_partial(const DevSystem &s, const DWork *work, int32_t w0, int32_t n_work, const double *n,
                              double *ne_part, cudaStream_t st);

// Records the text nao_last_error() returns on the calling thread (api.cpp).
void nao_set_last_error(const std::string &msg);

// ---- host helpers (partition.cpp) --------------------------------------------------------
// Recursive bisection (see nao_grid_create in nao.h); returns the number of batches.
int64_t nao_partition(int64_t n, const double *xyz, int64_t B, std::vector<int64_t> &offsets,
                      std::vector<int64_t> &perm);
// Natural cubic spline in the index coordinate: coefficients of y_k + c1 t + c2 t^2 + c3 t^3.
void nao_spline_coefficients(const double *y, int32_t n, double *coef /* [(n-1)*4] */);

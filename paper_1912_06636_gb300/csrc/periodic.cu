// Periodic systems (Eq. HamPeriodic, Eq. RealSpaceHamPeriodic, Eq. Bloch-basis).
//
// The real-space matrix h^uc is integrated over the unit cell's points with the same code as a
// finite system: the system's atoms are the periodic images R_A + T (T = n1 a1 + n2 a2 + n3 a3)
// whose functions can be non-zero in the cell, so its basis is the N_rs real-space functions of
// the paper. nao_periodic_images lists those images (host), nao_periodic_basis_map relates every
// image function to its unit-cell function and image, and nao_bloch_sum forms on the GPU
//     h_ij(k) = sum_{i' -> i, j' -> j} h^uc_{i'j'} e^{i k.(T_j' - T_i')},
// which is Eq. Bloch-basis, chi_ik = sum_T e^{i k.T} phi_i(r - T), inserted into Eq. HamPeriodic
// (conj(chi_i) on the left). The overlap s(k) follows from h^uc = S^uc (NAO_TERM_POTENTIAL, v = 1).
#include <cmath>
#include <string>
#include <vector>

#include "nao_internal.h"

namespace {

struct Lattice {
    double a[9];  // rows a1, a2, a3
};

// One thread per element (i', j') of h^uc for one k point (blockIdx.y); both the real and the
// imaginary part of e^{i k.(T_j' - T_i')} h^uc_{i'j'} are added into h(k)[fn(i')][fn(j')].
// The maps come from the caller: an element whose fn_map entry lies outside [0, nb) or whose
// fn_image entry lies outside [0, n_images) is skipped and counted in *err (when err is given),
// so that no map value can move a read or an atomic outside its array.
__global__ void __launch_bounds__(256) bloch_kernel(const double *__restrict__ huc, int64_t n_rs,
                                                   const int32_t *__restrict__ fn_map,
                                                   const int32_t *__restrict__ fn_image,
                                                   const int32_t *__restrict__ img_cell, int32_t n_images, Lattice L,
                                                   const double *__restrict__ kpts, int64_t nb, double *__restrict__ hk,
                                                   int32_t *__restrict__ err) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_rs * n_rs) return;
    const double hv = huc[e];
    if (hv == 0.0) return;
    const int64_t i = e / n_rs, j = e - i * n_rs;
    const int32_t mi = fn_map[i], mj = fn_map[j], ti = fn_image[i], tj = fn_image[j];
    if (mi < 0 || mi >= nb || mj < 0 || mj >= nb || ti < 0 || ti >= n_images || tj < 0 || tj >= n_images) {
        if (err && blockIdx.y == 0) atomicAdd(err, 1);
        return;
    }
    const int32_t *ci = img_cell + 3 * (int64_t)ti, *cj = img_cell + 3 * (int64_t)tj;
    const double *k = kpts + 3 * (int64_t)blockIdx.y;
    double ph = 0.0;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const double d = (double)(cj[0] - ci[0]) * L.a[c] + (double)(cj[1] - ci[1]) * L.a[3 + c] +
                         (double)(cj[2] - ci[2]) * L.a[6 + c];
        ph = fma(k[c], d, ph);
    }
    double sn, cs;
    sincos(ph, &sn, &cs);
    double *out = hk + 2 * (((int64_t)blockIdx.y * nb + mi) * nb + mj);
    atomicAdd(out, cs * hv);
    atomicAdd(out + 1, sn * hv);
}

bool inv3(const double *A, double *R) {
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    R[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    R[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    R[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    R[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    R[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    R[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    R[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    R[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    R[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    return true;
}

nao_status bad(nao_status s, const std::string &msg) {
    nao_set_last_error(msg);
    return s;
}

}  // namespace

extern "C" {

nao_status nao_periodic_images(const double *atom_xyz, int32_t n_atoms, const double *lattice, double reach,
                               int32_t max_images, double *img_xyz, int32_t *img_atom, int32_t *img_cell,
                               int32_t *n_images) {
    if (!atom_xyz || !lattice || !n_images || n_atoms <= 0 || !(reach >= 0.0) || max_images < 0)
        return bad(NAO_ERR_INVALID_ARG, "nao_periodic_images: bad argument");
    double Ainv[9];
    if (!inv3(lattice, Ainv)) return bad(NAO_ERR_INVALID_ARG, "nao_periodic_images: singular lattice");
    // fractional coordinates f = x Ainv (x = f A, rows of A are a1, a2, a3); the planes f_c =
    // const are 1 / |column c of Ainv| apart, so reach is m_c = reach |column c| in f_c
    double m[3];
    for (int c = 0; c < 3; c++)
        m[c] = reach * std::sqrt(Ainv[c] * Ainv[c] + Ainv[3 + c] * Ainv[3 + c] + Ainv[6 + c] * Ainv[6 + c]);
    const double eps = 1e-12;
    std::vector<double> xyz;
    std::vector<int32_t> atom, cell;
    for (int pass = 0; pass < 2; pass++)  // the atoms themselves (T = 0) first, then the other images
        for (int32_t a = 0; a < n_atoms; a++) {
            const double *x = atom_xyz + 3 * (int64_t)a;
            double f[3];
            for (int c = 0; c < 3; c++) f[c] = x[0] * Ainv[c] + x[1] * Ainv[3 + c] + x[2] * Ainv[6 + c];
            int lo[3], hi[3];
            for (int c = 0; c < 3; c++) {
                lo[c] = (int)std::floor(-m[c] - f[c]) - 1;
                hi[c] = (int)std::ceil(1.0 + m[c] - f[c]) + 1;
                if (hi[c] - lo[c] > 2000) return bad(NAO_ERR_INVALID_ARG, "nao_periodic_images: reach too large for the cell");
            }
            for (int n0 = lo[0]; n0 <= hi[0]; n0++)
                for (int n1 = lo[1]; n1 <= hi[1]; n1++)
                    for (int n2 = lo[2]; n2 <= hi[2]; n2++) {
                        const bool home = n0 == 0 && n1 == 0 && n2 == 0;
                        if ((pass == 0) != home) continue;
                        const int n[3] = {n0, n1, n2};
                        bool keep = true;
                        for (int c = 0; c < 3 && keep; c++) {
                            const double g = f[c] + n[c];
                            keep = g > -m[c] - eps && g < 1.0 + m[c] + eps;
                        }
                        if (!keep && !home) continue;
                        for (int c = 0; c < 3; c++)
                            xyz.push_back(x[c] + n0 * lattice[c] + n1 * lattice[3 + c] + n2 * lattice[6 + c]);
                        atom.push_back(a);
                        cell.push_back(n0);
                        cell.push_back(n1);
                        cell.push_back(n2);
                    }
        }
    *n_images = (int32_t)atom.size();
    if ((int64_t)atom.size() > max_images)
        return bad(NAO_ERR_INVALID_ARG, "nao_periodic_images: " + std::to_string(atom.size()) +
                                            " images exceed max_images (n_images holds the count)");
    if (!img_xyz || !img_atom || !img_cell) return bad(NAO_ERR_INVALID_ARG, "nao_periodic_images: NULL output");
    std::copy(xyz.begin(), xyz.end(), img_xyz);
    std::copy(atom.begin(), atom.end(), img_atom);
    std::copy(cell.begin(), cell.end(), img_cell);
    return NAO_OK;
}

nao_status nao_periodic_basis_map(const int32_t *atom_species, int32_t n_atoms, const int32_t *species_fn_offset,
                                  int32_t n_species, const int32_t *fn_l, const int32_t *img_atom, int32_t n_images,
                                  int64_t max_rs, int32_t *fn_map, int32_t *fn_image, int64_t *n_rs) {
    if (!atom_species || !species_fn_offset || !fn_l || !img_atom || !n_rs || n_atoms <= 0 || n_species <= 0 ||
        n_images < 0)
        return bad(NAO_ERR_INVALID_ARG, "nao_periodic_basis_map: bad argument");
    std::vector<int64_t> first(n_atoms + 1, 0);
    std::vector<int32_t> count(n_atoms, 0);
    for (int32_t a = 0; a < n_atoms; a++) {
        const int32_t sp = atom_species[a];
        if (sp < 0 || sp >= n_species) return bad(NAO_ERR_INVALID_ARG, "nao_periodic_basis_map: bad species");
        int32_t c = 0;
        for (int32_t f = species_fn_offset[sp]; f < species_fn_offset[sp + 1]; f++) c += 2 * fn_l[f] + 1;
        count[a] = c;
        first[a + 1] = first[a] + c;
    }
    int64_t total = 0;
    for (int32_t k = 0; k < n_images; k++) {
        if (img_atom[k] < 0 || img_atom[k] >= n_atoms) return bad(NAO_ERR_INVALID_ARG, "nao_periodic_basis_map: bad image atom");
        total += count[img_atom[k]];
    }
    *n_rs = total;
    if (total > max_rs) return bad(NAO_ERR_INVALID_ARG, "nao_periodic_basis_map: n_rs exceeds max_rs (n_rs holds the count)");
    if (!fn_map || !fn_image) return bad(NAO_ERR_INVALID_ARG, "nao_periodic_basis_map: NULL output");
    int64_t pos = 0;
    for (int32_t k = 0; k < n_images; k++) {
        const int32_t a = img_atom[k];
        for (int32_t t = 0; t < count[a]; t++, pos++) {
            fn_map[pos] = (int32_t)(first[a] + t);
            fn_image[pos] = k;
        }
    }
    return NAO_OK;
}

nao_status nao_bloch_sum(const double *h_uc_dev, int64_t n_rs, const int32_t *fn_map_dev, const int32_t *fn_image_dev,
                         const int32_t *img_cell_dev, int32_t n_images, const double *lattice, const double *k_dev,
                         int32_t n_k, int64_t nb, double *hk_dev, int32_t *err_dev, void *cuda_stream) {
    if (!h_uc_dev || !fn_map_dev || !fn_image_dev || !img_cell_dev || !lattice || !k_dev || !hk_dev || n_rs <= 0 ||
        n_k <= 0 || nb <= 0 || n_k > 65535 || n_images <= 0)
        return bad(NAO_ERR_INVALID_ARG, "nao_bloch_sum: bad argument");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    Lattice L;
    for (int c = 0; c < 9; c++) L.a[c] = lattice[c];
    cudaError_t e = cudaMemsetAsync(hk_dev, 0, 2 * (size_t)n_k * (size_t)nb * (size_t)nb * sizeof(double), st);
    if (e == cudaSuccess && err_dev) e = cudaMemsetAsync(err_dev, 0, sizeof(int32_t), st);
    const int64_t blocks = (n_rs * n_rs + 255) / 256;
    if (e == cudaSuccess && blocks > 0x7FFFFFFF) return bad(NAO_ERR_INVALID_ARG, "nao_bloch_sum: h^uc too large");
    if (e == cudaSuccess) {
        bloch_kernel<<<dim3((unsigned)blocks, (unsigned)n_k), 256, 0, st>>>(
            h_uc_dev, n_rs, fn_map_dev, fn_image_dev, img_cell_dev, n_images, L, k_dev, nb, hk_dev, err_dev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return bad(NAO_ERR_CUDA, std::string("nao_bloch_sum: ") + cudaGetErrorString(e));
    return NAO_OK;
}

}  // extern "C"

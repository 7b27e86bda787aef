// Host-side set-up steps of nao_grid_create: the batch partition and the radial splines.
#include <algorithm>
#include <cmath>

#include "nao_internal.h"

namespace {

struct Keyed {
    double key;
    int64_t idx;
};

inline bool keyed_less(const Keyed &a, const Keyed &b) { return a.key < b.key || (a.key == b.key && a.idx < b.idx); }

struct Splitter {
    const double *xyz;
    int64_t B;
    std::vector<Keyed> tmp;
    std::vector<int64_t> *perm;
    std::vector<int64_t> *offsets;

    // Batches leave in depth-first order. A leaf keeps the order its parent's cut gave it:
    // ascending (coordinate along the parent's axis, index); the root leaf keeps input order.
    void run(int64_t *S, int64_t n, int parent_axis) {
        const int64_t k = (n + B - 1) / B;
        if (k <= 1) {
            if (parent_axis >= 0) {
                for (int64_t i = 0; i < n; i++) tmp[i] = {xyz[3 * S[i] + parent_axis], S[i]};
                std::sort(tmp.begin(), tmp.begin() + n, keyed_less);
                for (int64_t i = 0; i < n; i++) S[i] = tmp[i].idx;
            }
            perm->insert(perm->end(), S, S + n);
            offsets->push_back((int64_t)perm->size());
            return;
        }
        double lo[3], hi[3];
        for (int c = 0; c < 3; c++) lo[c] = hi[c] = xyz[3 * S[0] + c];
        for (int64_t i = 1; i < n; i++)
            for (int c = 0; c < 3; c++) {
                const double v = xyz[3 * S[i] + c];
                lo[c] = v < lo[c] ? v : lo[c];
                hi[c] = v > hi[c] ? v : hi[c];
            }
        int ax = 0;
        for (int c = 1; c < 3; c++)
            if (hi[c] - lo[c] > hi[ax] - lo[ax]) ax = c;
        const int64_t nL = (n * (k / 2)) / k;
        for (int64_t i = 0; i < n; i++) tmp[i] = {xyz[3 * S[i] + ax], S[i]};
        // only the set that goes left matters here: the n_L smallest keys
        std::nth_element(tmp.begin(), tmp.begin() + nL, tmp.begin() + n, keyed_less);
        for (int64_t i = 0; i < n; i++) S[i] = tmp[i].idx;
        run(S, nL, ax);
        run(S + nL, n - nL, ax);
    }
};

}  // namespace

int64_t nao_partition(int64_t n, const double *xyz, int64_t B, std::vector<int64_t> &offsets,
                      std::vector<int64_t> &perm) {
    offsets.assign(1, 0);
    perm.clear();
    perm.reserve((size_t)n);
    std::vector<int64_t> S((size_t)n);
    for (int64_t i = 0; i < n; i++) S[(size_t)i] = i;
    Splitter sp{xyz, B, std::vector<Keyed>((size_t)n), &perm, &offsets};
    sp.run(S.data(), n, -1);
    return (int64_t)offsets.size() - 1;
}

// Natural cubic spline through (k, y_k): second derivatives from the tridiagonal system
// M_{k-1} + 4 M_k + M_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1}), M_0 = M_{n-1} = 0 (forward
// elimination, back substitution), then per segment the polynomial in t = s - k:
// y_k + c1 t + c2 t^2 + c3 t^3 with c1 = dy - (2 M_k + M_{k+1})/6, c2 = M_k/2,
// c3 = (M_{k+1} - M_k)/6.
void nao_spline_coefficients(const double *y, int32_t n, double *coef) {
    std::vector<double> M((size_t)n, 0.0), diag((size_t)n, 0.0), rhs((size_t)n, 0.0);
    for (int32_t k = 1; k < n - 1; k++) {
        diag[(size_t)k] = 4.0;
        rhs[(size_t)k] = 6.0 * (y[k + 1] - 2.0 * y[k] + y[k - 1]);
    }
    for (int32_t k = 2; k < n - 1; k++) {
        const double f = 1.0 / diag[(size_t)k - 1];
        diag[(size_t)k] -= f;
        rhs[(size_t)k] -= f * rhs[(size_t)k - 1];
    }
    for (int32_t k = n - 2; k >= 1; k--) {
        const double up = (k + 1 < n - 1) ? M[(size_t)k + 1] : 0.0;
        M[(size_t)k] = (rhs[(size_t)k] - up) / diag[(size_t)k];
    }
    for (int32_t k = 0; k < n - 1; k++) {
        double *c = coef + 4 * (size_t)k;
        c[0] = y[k];
        c[1] = (y[k + 1] - y[k]) - (2.0 * M[(size_t)k] + M[(size_t)k + 1]) / 6.0;
        c[2] = 0.5 * M[(size_t)k];
        c[3] = (M[(size_t)k + 1] - M[(size_t)k]) / 6.0;
    }
}

// C ABI of libnao (see include/nao.h): validation, set-up of a grid handle, and the
// per-call dispatch of the evaluation and contraction kernels onto the caller's stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>

#include "nao_internal.h"

namespace {

thread_local std::string g_last_error;

// Evaluation scratch when options.scratch_bytes is 0: 8 GiB (the split slices get three times as
// much). Each evaluation chunk is one launch of every kernel, so larger chunks mean fewer
// launches and fewer partly filled tails; memory is only taken up to what the handle's batches
// need.
constexpr int64_t kDefaultScratch = int64_t(8) << 30;


nao_status fail(nao_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

// ---- host-side fault injection ------------------------------------------------------------
// Tests how every entry point unwinds from a failed CUDA call without faulting a GPU: the n-th
// device allocation, host<->device copy or kernel launch counted from the setting fails, once,
// as if the CUDA call had returned an error (nothing is allocated, copied or launched for it).
// Set from the environment variable NAO_FAULT_INJECT ("alloc:<n>", "copy:<n>", "launch:<n>") when
// the library first needs it, or at run time by nao_fault_inject.
enum FaultKind { FAULT_NONE = 0, FAULT_ALLOC, FAULT_COPY, FAULT_LAUNCH };
struct FaultState {
    std::mutex mu;
    int kind = FAULT_NONE;
    int64_t n = 0, seen = 0;
};
thread_local bool g_fault_fired = false;  // the failure being reported was injected

bool parse_fault(const char *spec, int *kind, int64_t *n) {
    *kind = FAULT_NONE;
    *n = 0;
    if (!spec || !*spec) return true;
    const char *colon = std::strchr(spec, ':');
    if (!colon) return false;
    const std::string k(spec, colon - spec);
    char *end = nullptr;
    const long long v = std::strtoll(colon + 1, &end, 10);
    if (end == colon + 1 || *end != '\0' || v < 1) return false;
    if (k == "alloc") *kind = FAULT_ALLOC;
    else if (k == "copy") *kind = FAULT_COPY;
    else if (k == "launch") *kind = FAULT_LAUNCH;
    else return false;
    *n = v;
    return true;
}

FaultState &faults() {
    static FaultState *f = [] {
        FaultState *st = new FaultState();  // never destroyed: used until the process exits
        int kind;
        int64_t n;
        if (parse_fault(std::getenv("NAO_FAULT_INJECT"), &kind, &n)) {
            st->kind = kind;
            st->n = n;
        }
        return st;
    }();
    return *f;
}

// True (once) when this operation of the given kind is the one chosen to fail.
bool fault_fires(int kind) {
    FaultState &F = faults();
    std::lock_guard<std::mutex> lock(F.mu);
    if (F.kind != kind || ++F.seen < F.n) return false;
    F.kind = FAULT_NONE;
    g_fault_fired = true;
    return true;
}

nao_status cuda_fail(cudaError_t e, const char *what) {
    if (g_fault_fired) {
        g_fault_fired = false;
        return fail(NAO_ERR_CUDA, std::string("injected failure: ") + what);
    }
    return fail(NAO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define NAO_CUDA(expr)                                     \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
    } while (0)

// cudaMemcpyAsync, or the injected failure of a copy.
cudaError_t copy_async(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t st) {
    if (fault_fires(FAULT_COPY)) return cudaErrorInvalidValue;
    return cudaMemcpyAsync(dst, src, bytes, kind, st);
}

// Makes g's device current for the lifetime of the guard and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { prev = -1; ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// One memory pool per device for every handle's device memory. Stream-ordered allocation
// from it (cudaMallocFromPoolAsync / cudaFreeAsync on a handle's setup stream) neither waits
// for nor stalls work that other handles have in flight on other streams, which a serving loop
// that creates and destroys handles between other requests' launches relies on. The pool keeps
// freed memory for reuse while handles live; it is trimmed when the device's last handle goes.
struct PoolState {
    std::mutex mu;
    std::map<int, cudaMemPool_t> pool;
    std::map<int, int> live;
};
PoolState &pools() {
    static PoolState *p = new PoolState();  // never destroyed: handles may outlive static teardown
    return *p;
}

nao_status device_pool(int dev, cudaMemPool_t *out) {
    PoolState &P = pools();
    std::lock_guard<std::mutex> lock(P.mu);
    auto it = P.pool.find(dev);
    if (it == P.pool.end()) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        NAO_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = ~uint64_t(0);
        NAO_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        it = P.pool.emplace(dev, pool).first;
    }
    *out = it->second;
    return NAO_OK;
}

template <class T>
nao_status dev_alloc(nao_grid *g, T **p, size_t count) {
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaMemPool_t pool;
    nao_status st = device_pool(g->device, &pool);
    if (st) return st;
    if (fault_fires(FAULT_ALLOC)) {
        g_fault_fired = false;
        return fail(NAO_ERR_OUT_OF_MEMORY, "injected failure: device allocation of " + std::to_string(bytes) + " bytes");
    }
    const cudaError_t e = cudaMallocFromPoolAsync(&q, bytes, pool, g->setup);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NAO_ERR_OUT_OF_MEMORY, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    g->allocs.push_back(q);
    g->dev_bytes += (int64_t)bytes;
    *p = static_cast<T *>(q);
    return NAO_OK;
}

// Allocation plus an asynchronous copy on the setup stream; callers synchronise the setup
// stream before the memory is used from another stream (and before pageable sources die).
template <class T>
nao_status upload(nao_grid *g, T **p, const T *src, size_t count) {
    nao_status st = dev_alloc(g, p, count);
    if (st != NAO_OK) return st;
    if (count) NAO_CUDA(copy_async(*p, src, count * sizeof(T), cudaMemcpyHostToDevice, g->setup));
    return NAO_OK;
}

// Frees everything once the handle's last call has completed on the device, without waiting on
// the host for anything but this handle's own work.
void free_grid(nao_grid *g) {
    if (!g) return;
    if (g->setup && g->ev_last && g->used) cudaStreamWaitEvent(g->setup, g->ev_last, 0);
    if (!g->graphs.empty() && g->ev_last && g->used) cudaEventSynchronize(g->ev_last);
    for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
    for (auto &t : g->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : g->event_pool) cudaEventDestroy(e);
    if (g->ev_in) cudaEventDestroy(g->ev_in);
    if (g->ev_out) cudaEventDestroy(g->ev_out);
    if (g->gstream) cudaStreamDestroy(g->gstream);
    if (g->setup) {
        for (void *p : g->allocs) cudaFreeAsync(p, g->setup);
    }
    bool last = false;
    if (g->counted) {
        PoolState &P = pools();
        std::lock_guard<std::mutex> lock(P.mu);
        last = --P.live[g->device] == 0;
    }
    if (last) {
        // the device's last handle: return the pool's memory once these frees are done
        cudaStreamSynchronize(g->setup);
        cudaMemPool_t pool;
        if (device_pool(g->device, &pool) == NAO_OK) cudaMemPoolTrimTo(pool, 0);
    }
    if (g->ev_last) cudaEventDestroy(g->ev_last);
    if (g->setup) cudaStreamDestroy(g->setup);
    delete g;
}

// The handle's setup stream and last-call event (created first thing in nao_grid_create).
nao_status init_streams(nao_grid *g) {
    NAO_CUDA(cudaStreamCreateWithFlags(&g->setup, cudaStreamNonBlocking));
    NAO_CUDA(cudaEventCreateWithFlags(&g->ev_last, cudaEventDisableTiming));
    PoolState &P = pools();
    std::lock_guard<std::mutex> lock(P.mu);
    P.live[g->device]++;
    g->counted = true;
    return NAO_OK;
}

// Marks the end of a call's work on stream st.
nao_status mark_done(nao_grid *g, cudaStream_t st) {
    NAO_CUDA(cudaEventRecord(g->ev_last, st));
    g->used = true;
    return NAO_OK;
}

// Also marks the end of a call's work when the call returns early, after a failure part-way
// through its launches: the kernels it did enqueue are then still covered by ev_last, which
// destroy and nao_sync_status wait for before anything is freed or read. The failure's message
// is kept.
struct CallEnd {
    nao_grid *g;
    cudaStream_t st;
    CallEnd(nao_grid *g_, cudaStream_t s) : g(g_), st(s) {}
    ~CallEnd() {
        const std::string msg = g_last_error;
        if (cudaEventRecord(g->ev_last, st) == cudaSuccess) g->used = true;
        else cudaGetLastError();
        g_last_error = msg;
    }
};

double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; i++) f *= (double)i;
    return f;
}

inline bool finite(double x) { return std::isfinite(x); }

nao_status validate(const nao_system_desc *d, const nao_options &o) {
    if (!d) return fail(NAO_ERR_INVALID_ARG, "desc is NULL");
    if (d->n_atoms < 1 || !d->atom_xyz || !d->atom_species) return fail(NAO_ERR_INVALID_ARG, "no atoms");
    if (d->n_species < 1 || !d->species_fn_offset || !d->fn_l || !d->fn_cutoff || !d->fn_table)
        return fail(NAO_ERR_INVALID_ARG, "no species or radial functions");
    if (d->n_rgrid < 4) return fail(NAO_ERR_INVALID_ARG, "n_rgrid < 4");
    if (!(d->r0 > 0.0) || !(d->r_last > d->r0) || !finite(d->r_last)) return fail(NAO_ERR_INVALID_ARG, "bad r0/r_last");
    if (d->n_points < 1 || d->n_points >= (int64_t(1) << 31) || !d->pt_xyz || !d->pt_w)
        return fail(NAO_ERR_INVALID_ARG, "bad points");
    if (o.max_batch_points < 1 || o.max_batch_points > NAO_MAX_BATCH)
        return fail(NAO_ERR_INVALID_ARG, "max_batch_points must be in 1.." + std::to_string(NAO_MAX_BATCH));
    if (o.split_digits != NAO_DIGITS_BF16 && o.split_digits != NAO_DIGITS_E4M3)
        return fail(NAO_ERR_INVALID_ARG, "split_digits must be 0 (bf16) or 1 (e4m3)");
    if (o.split_digits == NAO_DIGITS_BF16 && (o.split_slices < 4 || o.split_slices > NAO_SPLIT_MAX_SLICES))
        return fail(NAO_ERR_INVALID_ARG, "split_slices must be in 4.." + std::to_string(NAO_SPLIT_MAX_SLICES) + " with bf16 digits");
    if (o.split_digits == NAO_DIGITS_E4M3 && (o.split_slices < 8 || o.split_slices > NAO_SPLIT_MAX_SLICES_E4M3))
        return fail(NAO_ERR_INVALID_ARG,
                    "split_slices must be in 8.." + std::to_string(NAO_SPLIT_MAX_SLICES_E4M3) + " with e4m3 digits");
    if (d->species_fn_offset[0] != 0) return fail(NAO_ERR_INVALID_ARG, "species_fn_offset[0] != 0");
    for (int s = 0; s < d->n_species; s++)
        if (d->species_fn_offset[s + 1] < d->species_fn_offset[s])
            return fail(NAO_ERR_INVALID_ARG, "species_fn_offset not ascending");
    const int n_fn = d->species_fn_offset[d->n_species];
    for (int f = 0; f < n_fn; f++) {
        if (d->fn_l[f] < 0 || d->fn_l[f] > NAO_LMAX) return fail(NAO_ERR_INVALID_ARG, "fn_l outside 0..6");
        if (!(d->fn_cutoff[f] > 0.0) || !(d->fn_cutoff[f] <= d->r_last))
            return fail(NAO_ERR_INVALID_ARG, "fn_cutoff outside (0, r_last]");
    }
    for (int64_t k = 0; k < (int64_t)n_fn * d->n_rgrid; k++)
        if (!finite(d->fn_table[k])) return fail(NAO_ERR_INVALID_ARG, "non-finite fn_table entry");
    for (int a = 0; a < d->n_atoms; a++) {
        if (d->atom_species[a] < 0 || d->atom_species[a] >= d->n_species)
            return fail(NAO_ERR_INVALID_ARG, "atom_species out of range");
        for (int c = 0; c < 3; c++)
            if (!finite(d->atom_xyz[3 * a + c])) return fail(NAO_ERR_INVALID_ARG, "non-finite atom coordinate");
    }
    for (int64_t p = 0; p < d->n_points; p++) {
        if (!finite(d->pt_xyz[3 * p]) || !finite(d->pt_xyz[3 * p + 1]) || !finite(d->pt_xyz[3 * p + 2]) ||
            !finite(d->pt_w[p]))
            return fail(NAO_ERR_INVALID_ARG, "non-finite point or weight");
    }
    return NAO_OK;
}

// One or more systems concatenated: atoms, radial functions and points get global indices;
// each system is partitioned on its own, so no batch mixes systems.
nao_status build(nao_grid *g, const nao_system_desc *descs, int32_t n_sys, const int32_t *batch_points) {
    const nao_system_desc *d0 = &descs[0];
    g->n_sys = n_sys;
    g->n_rgrid = d0->n_rgrid;
    g->r0 = d0->r0;
    g->r_last = d0->r_last;
    g->delta = std::log(d0->r_last / d0->r0) / (double)(d0->n_rgrid - 1);

    // global atoms, radial functions and points
    std::vector<double> atoms, fn_cut, fn_tab;
    std::vector<int32_t> atom_fn0, atom_fn1, fn_l;
    std::vector<int64_t> atom_basis(1, 0);
    std::vector<double> pts, wts;
    g->sys_boff.assign(n_sys, 0);
    g->sys_nb.assign(n_sys, 0);
    g->sys_poff.assign(n_sys, 0);
    g->sys_np.assign(n_sys, 0);
    g->sys_aoff.assign(n_sys + 1, 0);
    int32_t fn_base = 0;
    for (int m = 0; m < n_sys; m++) {
        const nao_system_desc *d = &descs[m];
        if (d->n_rgrid != d0->n_rgrid || d->r0 != d0->r0 || d->r_last != d0->r_last)
            return fail(NAO_ERR_INVALID_ARG, "systems of one handle must share n_rgrid, r0 and r_last");
        const int nfn = d->species_fn_offset[d->n_species];
        for (int f = 0; f < nfn; f++) {
            fn_l.push_back(d->fn_l[f]);
            fn_cut.push_back(d->fn_cutoff[f]);
        }
        fn_tab.insert(fn_tab.end(), d->fn_table, d->fn_table + (size_t)nfn * d->n_rgrid);
        g->sys_boff[m] = (int32_t)atom_basis.back();
        g->sys_aoff[m] = (int32_t)(atoms.size() / 3);
        for (int a = 0; a < d->n_atoms; a++) {
            const int sp = d->atom_species[a];
            int64_t c = 0;
            for (int f = d->species_fn_offset[sp]; f < d->species_fn_offset[sp + 1]; f++) c += 2 * d->fn_l[f] + 1;
            atoms.insert(atoms.end(), d->atom_xyz + 3 * a, d->atom_xyz + 3 * a + 3);
            atom_fn0.push_back(fn_base + d->species_fn_offset[sp]);
            atom_fn1.push_back(fn_base + d->species_fn_offset[sp + 1]);
            atom_basis.push_back(atom_basis.back() + c);
        }
        g->sys_aoff[m + 1] = (int32_t)(atoms.size() / 3);
        g->sys_nb[m] = (int32_t)(atom_basis.back() - g->sys_boff[m]);
        if (g->sys_nb[m] < 1) return fail(NAO_ERR_INVALID_ARG, "a system has no basis functions");
        g->sys_poff[m] = (int32_t)(pts.size() / 3);
        g->sys_np[m] = (int32_t)d->n_points;
        pts.insert(pts.end(), d->pt_xyz, d->pt_xyz + 3 * d->n_points);
        wts.insert(wts.end(), d->pt_w, d->pt_w + d->n_points);
        fn_base += nfn;
        if ((int64_t)pts.size() / 3 >= (int64_t(1) << 31)) return fail(NAO_ERR_INVALID_ARG, "too many points");
    }
    g->n_atoms = (int32_t)(atoms.size() / 3);
    g->n_fn = fn_base;
    g->nb = atom_basis.back();
    if (g->nb >= (int64_t(1) << 31)) return fail(NAO_ERR_INVALID_ARG, "too many basis functions");
    g->atom_basis.assign(atom_basis.begin(), atom_basis.end());
    const int64_t n = (int64_t)wts.size();
    g->n_points = n;

    // Sec. 3.3.1: batches, system by system. The systems' partitions are independent, so they
    // run on host threads (each system on one thread, systems handed out in order of size);
    // the result is the same as in sequence.
    std::vector<int32_t> bmol;
    g->batch_off.assign(1, 0);
    g->perm.clear();
    for (int m = 0; m < n_sys; m++) {
        const int B = batch_points ? batch_points[m] : g->opt.max_batch_points;
        if (B < 1 || B > NAO_MAX_BATCH) return fail(NAO_ERR_INVALID_ARG, "batch size outside 1..1024");
    }
    std::vector<std::vector<int64_t>> offs(n_sys), perms(n_sys);
    {
        std::vector<int32_t> order(n_sys);
        for (int m = 0; m < n_sys; m++) order[m] = m;
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return descs[a].n_points > descs[b].n_points; });
        std::atomic<int32_t> next{0};
        auto work = [&]() {
            for (int32_t k; (k = next.fetch_add(1)) < n_sys;) {
                const int m = order[k];
                nao_partition(descs[m].n_points, descs[m].pt_xyz, batch_points ? batch_points[m] : g->opt.max_batch_points,
                              offs[m], perms[m]);
            }
        };
        int64_t total_pts = 0;
        for (int m = 0; m < n_sys; m++) total_pts += descs[m].n_points;
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nthr = (int)std::min<int64_t>({(int64_t)hw, (int64_t)n_sys, 1 + total_pts / 200000});
        std::vector<std::thread> pool;
        try {
            for (int t = 1; t < nthr; t++) pool.emplace_back(work);
        } catch (...) {  // no more threads: the calling thread does the rest
        }
        work();
        for (auto &th : pool) th.join();
    }
    for (int m = 0; m < n_sys; m++) {
        const std::vector<int64_t> &off = offs[m];
        for (size_t k = 1; k < off.size(); k++) {
            g->batch_off.push_back(g->sys_poff[m] + off[k]);
            bmol.push_back(m);
        }
        for (int64_t p : perms[m]) g->perm.push_back(g->sys_poff[m] + p);
        std::vector<int64_t>().swap(offs[m]);
        std::vector<int64_t>().swap(perms[m]);
    }
    g->n_batches = (int64_t)bmol.size();
    const int64_t nbat = g->n_batches;

    // points in batch order, structure of arrays
    std::vector<double> px(n), py(n), pz(n), pw(n);
    std::vector<int32_t> perm32(n), boff32(nbat + 1);
    for (int64_t i = 0; i < n; i++) {
        const int64_t p = g->perm[i];
        px[i] = pts[3 * p];
        py[i] = pts[3 * p + 1];
        pz[i] = pts[3 * p + 2];
        pw[i] = wts[p];
        perm32[i] = (int32_t)p;
    }
    for (int64_t b = 0; b <= nbat; b++) boff32[b] = (int32_t)g->batch_off[b];

    nao_status st;
    double *d_px, *d_py, *d_pz, *d_pw, *d_atoms;
    int32_t *d_perm, *d_boff, *d_bmol, *d_aoff;
    if ((st = upload(g, &d_px, px.data(), n)) || (st = upload(g, &d_py, py.data(), n)) ||
        (st = upload(g, &d_pz, pz.data(), n)) || (st = upload(g, &d_pw, pw.data(), n)) ||
        (st = upload(g, &d_perm, perm32.data(), n)) || (st = upload(g, &d_boff, boff32.data(), nbat + 1)) ||
        (st = upload(g, &d_atoms, atoms.data(), atoms.size())) || (st = upload(g, &d_bmol, bmol.data(), bmol.size())) ||
        (st = upload(g, &d_aoff, g->sys_aoff.data(), g->sys_aoff.size())))
        return st;

    // Sec. 3.3.2: nnz(B) from the per-(batch, atom of its system) minimum distance
    int32_t max_atoms = 0;
    for (int m = 0; m < n_sys; m++) max_atoms = std::max(max_atoms, g->sys_aoff[m + 1] - g->sys_aoff[m]);
    std::vector<double> minr2((size_t)nbat * max_atoms);
    {
        double *d_minr2;
        if ((st = dev_alloc(g, &d_minr2, minr2.size()))) return st;
        NAO_CUDA(launch_relevance_minr2(d_atoms, d_bmol, d_aoff, max_atoms, d_px, d_py, d_pz, d_boff, nbat, d_minr2,
                                        g->setup));
        NAO_CUDA(copy_async(minr2.data(), d_minr2, minr2.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                 g->setup));
        NAO_CUDA(cudaStreamSynchronize(g->setup));
        cudaFreeAsync(d_minr2, g->setup);
        g->allocs.pop_back();
        g->dev_bytes -= (int64_t)std::max<size_t>(minr2.size() * sizeof(double), 16);
    }

    std::vector<RfnEntry> rfn;
    std::vector<int32_t> rfn_off32(nbat + 1, 0), rel_off32(nbat + 1, 0);
    g->rel_off.assign(nbat + 1, 0);
    g->Pb.resize(nbat);
    g->Nb.resize(nbat);
    for (int64_t b = 0; b < nbat; b++) {
        const int m = bmol[b];
        int32_t pos = 0;
        for (int a = g->sys_aoff[m]; a < g->sys_aoff[m + 1]; a++) {
            const double m2 = minr2[(size_t)b * max_atoms + (a - g->sys_aoff[m])];
            if (m2 == 0.0) return fail(NAO_ERR_INVALID_ARG, "a grid point coincides with a nucleus");
            int64_t base = atom_basis[a];
            for (int f = atom_fn0[a]; f < atom_fn1[a]; f++) {
                const int l = fn_l[f];
                const double rc = fn_cut[f];
                if (m2 < rc * rc) {
                    rfn.push_back({a, f, pos, l});
                    for (int q = 0; q < 2 * l + 1; q++) g->rel_idx.push_back((int32_t)(base + q));
                    pos += 2 * l + 1;
                }
                base += 2 * l + 1;
            }
        }
        g->rel_off[b + 1] = (int64_t)g->rel_idx.size();
        rfn_off32[b + 1] = (int32_t)rfn.size();
        g->Pb[b] = (int32_t)(g->batch_off[b + 1] - g->batch_off[b]);
        g->Nb[b] = pos;
        g->max_P = std::max(g->max_P, g->Pb[b]);
        g->max_N = std::max(g->max_N, pos);
        const double P = g->Pb[b], N = pos;
        g->flops_h += (int64_t)(4.0 * P * N * (N + 1.0));
        g->flops_n += (int64_t)(2.0 * P * N * N + 2.0 * P * N);
    }
    g->rel_total = (int64_t)g->rel_idx.size();
    g->rfn_total = (int64_t)rfn.size();
    // atom groups: consecutive entries of one atom, sorted by l (positions are kept)
    std::vector<AtomGroup> agrp;
    std::vector<int32_t> agrp_off32(nbat + 1, 0);
    for (int64_t b = 0; b < nbat; b++) {
        int32_t i = rfn_off32[b];
        while (i < rfn_off32[b + 1]) {
            int32_t j = i;
            while (j < rfn_off32[b + 1] && rfn[j].atom == rfn[i].atom) j++;
            std::stable_sort(rfn.begin() + i, rfn.begin() + j,
                             [](const RfnEntry &x, const RfnEntry &y) { return x.l < y.l; });
            agrp.push_back({rfn[i].atom, i, j - i, rfn[j - 1].l});
            i = j;
        }
        agrp_off32[b + 1] = (int32_t)agrp.size();
    }
    if (g->rel_total >= (int64_t(1) << 31)) return fail(NAO_ERR_UNSUPPORTED, "reduced bases too large");
    for (int64_t b = 0; b <= nbat; b++) rel_off32[b] = (int32_t)g->rel_off[b];

    // radial splines
    const int nr = g->n_rgrid;
    std::vector<double> coef((size_t)g->n_fn * (nr - 1) * 4);
    for (int f = 0; f < g->n_fn; f++)
        nao_spline_coefficients(fn_tab.data() + (size_t)f * nr, nr, coef.data() + (size_t)f * (nr - 1) * 4);
    std::vector<float> coef32(coef.begin(), coef.end()), coef_lo(coef.size());
    for (size_t q = 0; q < coef.size(); q++) coef_lo[q] = (float)(coef[q] - (double)coef32[q]);
    // Segments whose cubic is ill-conditioned (coefficient magnitudes above 4x the smaller end
    // value, or above 4x the smaller end slope: the decaying tails of steep functions, the
    // approach to the cutoff, extrema) lose more than a few FP32 ulps to cancellation; the FP32
    // path evaluates them from the FP64 coefficients.
    std::vector<uint8_t> seg64((size_t)g->n_fn * (nr - 1), 0);
    for (size_t q = 0; q < seg64.size(); q++) {
        const double *c = coef.data() + 4 * q;
        const double y0 = std::fabs(c[0]), y1 = std::fabs(c[0] + c[1] + c[2] + c[3]);
        const double d0 = std::fabs(c[1]), d1 = std::fabs(c[1] + 2.0 * c[2] + 3.0 * c[3]);
        const double sv = std::fabs(c[0]) + std::fabs(c[1]) + std::fabs(c[2]) + std::fabs(c[3]);
        const double sd = std::fabs(c[1]) + 2.0 * std::fabs(c[2]) + 3.0 * std::fabs(c[3]);
        seg64[q] = (sv > 4.0 * std::min(y0, y1) || sd > 4.0 * std::min(d0, d1)) ? 1 : 0;
    }
    std::vector<double> inv_rk((size_t)nr);
    for (int k = 0; k < nr; k++) inv_rk[(size_t)k] = 1.0 / (g->r0 * std::exp((double)k * g->delta));

    // work lists and chunks of batches that fit the scratch
    std::vector<HWork> hw;
    std::vector<DWork> dw;
    std::vector<int64_t> scr_off(nbat, 0);
    int64_t budget = (g->opt.scratch_bytes > 0 ? g->opt.scratch_bytes : kDefaultScratch) / (int64_t)sizeof(double);
    int64_t need_max = 0, need_total = 0;
    for (int64_t b = 0; b < nbat; b++) {
        const int64_t Ppad = (g->Pb[b] + NAO_PPAD - 1) / NAO_PPAD * NAO_PPAD;
        const int64_t e = (int64_t)g->Nb[b] * 4 * Ppad;
        need_max = std::max(need_max, e);
        need_total += e;
    }
    budget = std::max(budget, need_max);
    budget = std::min(budget, std::max<int64_t>(need_total, 16));
    Chunk cur{0, 0, 0, 0, 0, 0};
    int64_t used = 0;
    for (int64_t b = 0; b < nbat; b++) {
        const int64_t Ppad = (g->Pb[b] + NAO_PPAD - 1) / NAO_PPAD * NAO_PPAD;
        const int64_t e = (int64_t)g->Nb[b] * 4 * Ppad;
        if (used + e > budget && b > cur.b0) {
            cur.b1 = (int32_t)b;
            cur.hw1 = (int32_t)hw.size();
            cur.dw1 = (int32_t)dw.size();
            g->chunks.push_back(cur);
            cur = Chunk{(int32_t)b, 0, (int32_t)hw.size(), 0, (int32_t)dw.size(), 0};
            used = 0;
        }
        scr_off[b] = used;
        used += e;
        const int nt = (g->Nb[b] + NAO_TILE - 1) / NAO_TILE;
        for (int i = 0; i < nt; i++)
            for (int j = i; j < nt; j++) hw.push_back({(int32_t)b, i, j, 0});
        const int np = (g->Pb[b] + NAO_TILE - 1) / NAO_TILE;
        for (int t = 0; t < np; t++) dw.push_back({(int32_t)b, t});
    }
    cur.b1 = (int32_t)nbat;
    cur.hw1 = (int32_t)hw.size();
    cur.dw1 = (int32_t)dw.size();
    g->chunks.push_back(cur);
    g->scratch_elems = budget;
    g->n_hwork = (int64_t)hw.size();
    g->n_dwork = (int64_t)dw.size();
    // per system: density items, H zeroing chunks and mirror tiles
    g->sys_dw0.assign(n_sys + 1, 0);
    for (int64_t w = 0; w < g->n_dwork; w++) g->sys_dw0[bmol[dw[w].batch] + 1] = (int32_t)(w + 1);
    for (int m = 0; m < n_sys; m++) g->sys_dw0[m + 1] = std::max(g->sys_dw0[m + 1], g->sys_dw0[m]);
    for (int m = 0; m < n_sys; m++) {
        const int64_t tot = (int64_t)g->sys_nb[m] * g->sys_nb[m];
        for (int64_t c = 0; c * 65536 < tot; c++)
            g->zero_tasks.push_back(make_int4(m, (int)c, (int)std::min<int64_t>(65536, tot - c * 65536), 0));
        const int nt = (g->sys_nb[m] + 31) / 32;
        for (int bx = 0; bx < nt; bx++)
            for (int by = 0; by <= bx; by++) g->mirror_tasks.push_back(make_int4(m, bx, by, 0));
    }

    double *d_coef, *d_rc;
    float *d_coef32, *d_coef_lo;
    double *d_inv_rk;
    int32_t *d_rel_off, *d_rel_idx, *d_rfn_off;
    RfnEntry *d_rfn;
    AtomGroup *d_agrp;
    int32_t *d_agrp_off;
    int64_t *d_scr_off;
    uint8_t *d_seg64;
    if ((st = upload(g, &d_coef, coef.data(), coef.size())) || (st = upload(g, &d_coef32, coef32.data(), coef32.size())) ||
        (st = upload(g, &d_coef_lo, coef_lo.data(), coef_lo.size())) ||
        (st = upload(g, &d_seg64, seg64.data(), seg64.size())) ||
        (st = upload(g, &d_inv_rk, inv_rk.data(), inv_rk.size())) ||
        (st = upload(g, &d_rc, fn_cut.data(), fn_cut.size())) ||
        (st = upload(g, &d_rel_off, rel_off32.data(), rel_off32.size())) ||
        (st = upload(g, &d_rel_idx, g->rel_idx.data(), g->rel_idx.size())) ||
        (st = upload(g, &d_rfn_off, rfn_off32.data(), rfn_off32.size())) ||
        (st = upload(g, &d_rfn, rfn.data(), rfn.size())) || (st = upload(g, &d_scr_off, scr_off.data(), scr_off.size())) ||
        (st = upload(g, &d_agrp, agrp.data(), agrp.size())) ||
        (st = upload(g, &d_agrp_off, agrp_off32.data(), agrp_off32.size())) ||
        (st = upload(g, &g->d_hwork, hw.data(), hw.size())) || (st = upload(g, &g->d_dwork, dw.data(), dw.size())) ||
        (st = dev_alloc(g, &g->d_scratch, (size_t)g->scratch_elems)) ||
        (st = dev_alloc(g, &g->d_ne_part, (size_t)std::max<int64_t>(g->n_dwork, 1))) ||
        (st = dev_alloc(g, &g->d_err, 4)))
        return st;
    NAO_CUDA(cudaMemsetAsync(g->d_err, 0, 4 * sizeof(int32_t), g->setup));
    int32_t *d_sboff, *d_snb, *d_spoff;
    if ((st = upload(g, &d_sboff, g->sys_boff.data(), g->sys_boff.size())) ||
        (st = upload(g, &d_snb, g->sys_nb.data(), g->sys_nb.size())) ||
        (st = upload(g, &d_spoff, g->sys_poff.data(), g->sys_poff.size())) ||
        (st = upload(g, &g->d_sys_dw0, g->sys_dw0.data(), g->sys_dw0.size())) ||
        (st = upload(g, &g->d_zero_tasks, g->zero_tasks.data(), g->zero_tasks.size())) ||
        (st = upload(g, &g->d_mirror_tasks, g->mirror_tasks.data(), g->mirror_tasks.size())) ||
        (st = upload(g, &g->d_sys_np, g->sys_np.data(), g->sys_np.size())) ||
        (st = dev_alloc(g, &g->d_tab, 8 * (size_t)n_sys)))
        return st;
    NAO_CUDA(cudaMemsetAsync(g->d_tab, 0, 8 * (size_t)n_sys * sizeof(double *), g->setup));
    g->h_tab.assign(8 * (size_t)n_sys, nullptr);
    if (g->opt.deterministic) {
        // section 7: each system's fixed-point H accumulators (2 words per element), fixed for the
        // handle's life
        for (int m = 0; m < n_sys; m++) {
            unsigned long long *acc = nullptr;
            if ((st = dev_alloc(g, &acc, 2 * (size_t)g->sys_nb[m] * (size_t)g->sys_nb[m]))) return st;
            g->h_tab[7 * (size_t)n_sys + m] = acc;
        }
        NAO_CUDA(copy_async(g->d_tab + 7 * (size_t)n_sys, g->h_tab.data() + 7 * (size_t)n_sys,
                            (size_t)n_sys * sizeof(void *), cudaMemcpyHostToDevice, g->setup));
    }

    DevSystem &s = g->sys;
    s.atom_xyz = d_atoms;
    s.coef = d_coef;
    s.coef_f32 = d_coef32;
    s.coef_lo = d_coef_lo;
    s.inv_rk = d_inv_rk;
    s.seg64 = d_seg64;
    s.fn_rc = d_rc;
    s.px = d_px;
    s.py = d_py;
    s.pz = d_pz;
    s.pw = d_pw;
    s.perm = d_perm;
    s.batch_off = d_boff;
    s.rel_off = d_rel_off;
    s.rel_idx = d_rel_idx;
    s.rfn_off = d_rfn_off;
    s.rfn = d_rfn;
    s.agrp = d_agrp;
    s.agrp_off = d_agrp_off;
    s.scr_off = d_scr_off;
    s.sys.bmol = d_bmol;
    s.sys.boff = d_sboff;
    s.sys.nbm = d_snb;
    s.sys.poff = d_spoff;
    s.sys.aoff = d_aoff;
    s.sys.H = g->d_tab;
    s.sys.v = g->d_tab + n_sys;
    s.sys.P = g->d_tab + 2 * n_sys;
    s.sys.n = g->d_tab + 3 * n_sys;
    s.sys.ne = g->d_tab + 4 * n_sys;
    s.sys.gn = g->d_tab + 5 * n_sys;
    s.sys.vt = g->d_tab + 6 * n_sys;
    s.sys.Hacc = reinterpret_cast<unsigned long long *const *>(g->d_tab + 7 * n_sys);
    s.sys.np = g->d_sys_np;
    s.n_rgrid = g->n_rgrid;
    s.r0 = g->r0;
    s.inv_delta = 1.0 / g->delta;
    s.step_m1 = std::expm1(g->delta);
    s.nb = g->nb;
    for (int l = 0; l <= NAO_LMAX; l++)
        for (int m = 0; m <= NAO_LMAX; m++) {
            double k = 0.0;
            if (m <= l) {
                k = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
                if (m > 0) k *= std::sqrt(2.0);
            }
            s.knorm[l][m] = k;
            s.knorm_h[l][m] = (float)k;
            s.knorm_l[l][m] = (float)(k - (double)s.knorm_h[l][m]);
        }
    NAO_CUDA(cudaStreamSynchronize(g->setup));
    return NAO_OK;
}

cudaEvent_t take_event(nao_grid *g) {
    if (!g->event_pool.empty()) {
        cudaEvent_t e = g->event_pool.back();
        g->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Runs one launcher; when profiling, brackets it with events on the stream.
template <class F>
cudaError_t timed(nao_grid *g, int kid, cudaStream_t st, F &&launch) {
    if (fault_fires(FAULT_LAUNCH)) return cudaErrorLaunchFailure;
    if (!g->profiling) return launch();
    cudaEvent_t a = take_event(g), b = take_event(g);
    if (!a || !b) return launch();
    cudaEventRecord(a, st);
    const cudaError_t e = launch();
    cudaEventRecord(b, st);
    g->timed.push_back({kid, a, b});
    return e;
}

nao_status check_handle(const nao_grid *g) {
    if (!g) return fail(NAO_ERR_INVALID_ARG, "handle is NULL");
    return NAO_OK;
}

nao_status check_prec(nao_precision p) {
    if (p != NAO_FP64 && p != NAO_FP32 && p != NAO_SPLIT) return fail(NAO_ERR_INVALID_ARG, "unknown precision");
    return NAO_OK;
}

// Split-path tile width of a batch before (or without) autotuning: 32 where 48 cannot hold
// the S accumulator groups in tensor memory, else 48 (every width in use costs a launch of its
// own, so small batches stay with the majority).
int default_tn(int S, int F) { return nao_split_tn(S, F); }

// The split work lists for the current per-batch tile widths, per split chunk and width:
// H tile pairs (batch, 128-row tile I, TN-column tile J) crossing the upper triangle, and
// density items (batch, 128-point tile, number of TN-function tiles).
nao_status split_lists(nao_grid *g) {
    const int S = g->split_S, F = g->split_F;
    g->split_lists_ver++;
    std::vector<HWork> hw[2], nw[2];
    for (auto &c : g->split_chunks) {
        for (int k = 0; k < 2; k++) {
            c.hw0[k] = (int32_t)hw[k].size();
            c.nw0[k] = (int32_t)nw[k].size();
        }
        for (int32_t b = c.b0; b < c.b1; b++) {
            const int P = g->Pb[b], N = g->Nb[b];
            if (N == 0) continue;
            const int TN = g->split_tn[b], k = TN == 48 ? 0 : 1;
            const SplitGeom G(P, N, S, TN, F);
            nao_split_h_items(b, P, N, TN, S, hw[k], F);
            for (int Q = 0; Q < G.n_qt; Q++) nw[k].push_back({b, Q, G.n_jtN, 0});  // all J tiles in one CTA
        }
        // the persistent contraction kernels take items round-robin: heaviest first (H: longest
        // K, i.e. most K chunks in the item's segment; density: most function tiles), so that
        // every CTA gets a similar share
        auto item_kc = [&](const HWork &x) {
            const SplitGeom G(g->Pb[x.batch], g->Nb[x.batch], S, 0, F);
            int kc0, kc1;
            nao_split_h_seg_range(G.n_kc, nao_split_h_nseg(g->Pb[x.batch], S, F), x.pad, S, kc0, kc1, F);
            return kc1 - kc0;
        };
        for (int k = 0; k < 2; k++) {
            std::stable_sort(hw[k].begin() + c.hw0[k], hw[k].end(),
                             [&](const HWork &x, const HWork &y) { return item_kc(x) > item_kc(y); });
            std::stable_sort(nw[k].begin() + c.nw0[k], nw[k].end(),
                             [](const HWork &x, const HWork &y) { return x.tj > y.tj; });
            c.hw1[k] = (int32_t)hw[k].size();
            c.nw1[k] = (int32_t)nw[k].size();
        }
    }
    // one array per list: width-48 items, then width-32 items (offsets shifted below)
    const int64_t nh = (int64_t)(hw[0].size() + hw[1].size()), nn = (int64_t)(nw[0].size() + nw[1].size());
    if (nh > g->cap_split_hw || nn > g->cap_split_nw)
        return fail(NAO_ERR_INTERNAL, "split work lists exceed their planned capacity");
    for (auto &c : g->split_chunks) {
        c.hw0[1] += (int32_t)hw[0].size();
        c.hw1[1] += (int32_t)hw[0].size();
        c.nw0[1] += (int32_t)nw[0].size();
        c.nw1[1] += (int32_t)nw[0].size();
    }
    hw[0].insert(hw[0].end(), hw[1].begin(), hw[1].end());
    nw[0].insert(nw[0].end(), nw[1].begin(), nw[1].end());
    if (!hw[0].empty())
        NAO_CUDA(copy_async(g->d_split_hw, hw[0].data(), hw[0].size() * sizeof(HWork), cudaMemcpyHostToDevice, g->setup));
    if (!nw[0].empty())
        NAO_CUDA(copy_async(g->d_split_nw, nw[0].data(), nw[0].size() * sizeof(HWork), cudaMemcpyHostToDevice, g->setup));
    NAO_CUDA(copy_async(g->d_split_tn, g->split_tn.data(), g->split_tn.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, g->setup));
    NAO_CUDA(cudaStreamSynchronize(g->setup));
    g->n_split_hw = nh;
    g->n_split_nw = nn;
    // recorded graphs hold the old lists' launch ranges
    if (!g->graphs.empty()) {
        if (g->gstream) NAO_CUDA(cudaStreamSynchronize(g->gstream));
        for (auto &kv : g->graphs) cudaGraphExecDestroy(kv.second);
        g->graphs.clear();
    }
    return NAO_OK;
}

// Plan and allocate the split path: sub-chunks of the evaluation chunks whose slices fit the
// slice budget, per-batch slice offsets and exponent arrays, work lists.
nao_status split_setup(nao_grid *g) {
    if (g->split_ready) return NAO_OK;
    const int S = g->opt.split_slices, F = g->opt.split_digits;
    if (S > (F == NAO_DIGITS_E4M3 ? NAO_SPLIT_MAX_SLICES_E4M3 : NAO_SPLIT_MAX_SLICES))
        return fail(NAO_ERR_UNSUPPORTED, "too many slices for the split path's tensor memory");
    const int C = nao_chunk_cols(F);
    for (int64_t b = 0; b < g->n_batches; b++) {
        const int64_t Ppad = (g->Pb[b] + NAO_PPAD - 1) / NAO_PPAD * NAO_PPAD;
        const int64_t N64 = (g->Nb[b] + C - 1) / C * C;
        // every slice-group sum must stay below 2^24: K S 2^(2 bits - 2) < 2^24. The H
        // contraction (K = 4 Ppad) splits K into segments where needed; the density's K is the
        // batch's basis (N rounded up to a K chunk), one accumulation per function tile
        if (Ppad > NAO_SPLIT_MAX_PPAD)
            return fail(NAO_ERR_UNSUPPORTED, "batch too large for the split path (points " + std::to_string(g->Pb[b]) +
                                                 ", at most " + std::to_string(NAO_SPLIT_MAX_PPAD) + ")");
        if (N64 * S >= nao_exact_ks(F))
            return fail(NAO_ERR_UNSUPPORTED, "batch too large for exact slice sums (basis " + std::to_string(g->Nb[b]) +
                                                 ", slices " + std::to_string(S) + ")");
    }
    NAO_CUDA(split_configure());
    g->split_chunks.clear();  // a failed earlier set-up may have planned part of them
    // slices take S x 2 (bf16) or S (e4m3) bytes per evaluated FP64 value (8 bytes): three times
    // the evaluation budget holds one evaluation chunk's slices at up to 12 bf16 or 16 e4m3 slices
    const int64_t budget =
        std::max<int64_t>(3 * (g->opt.scratch_bytes > 0 ? g->opt.scratch_bytes : kDefaultScratch), int64_t(1) << 20);
    std::vector<int64_t> off_h(g->n_batches, 0), off_n(g->n_batches, 0);
    int64_t max_used = 0, cap_h = 0, cap_n = 0;
    g->split_tn.assign(g->n_batches, 32);
    for (const Chunk &c : g->chunks) {
        nao_grid::SplitChunk cur{};
        cur.b0 = cur.b1 = c.b0;
        int64_t used = 0;
        for (int32_t b = c.b0; b < c.b1; b++) {
            const int P = g->Pb[b], N = g->Nb[b];
            const SplitGeom G(P, N, S, 0, F);
            const int64_t need = N == 0 ? 0 : (int64_t)std::max(G.h_bytes(S), G.n_bytes(S));
            if (used + need > budget && b > cur.b0) {
                cur.b1 = b;
                g->split_chunks.push_back(cur);
                cur = nao_grid::SplitChunk{};
                cur.b0 = cur.b1 = b;
                used = 0;
            }
            off_h[b] = used;
            off_n[b] = used;
            used += need;
            max_used = std::max(max_used, used);
            g->split_tn[b] = default_tn(S, F);
            if (N > 0) {
                cur.max_rt = std::max<int32_t>(cur.max_rt, G.h_slice_tiles());
                cur.max_qt = std::max<int32_t>(cur.max_qt, G.n_qt);
                // list capacity: the larger of the two widths' item counts
                int64_t best_h = 0;
                for (int TN : {48, 32}) {
                    if (TN == 48 && nao_split_tn(S, F) != 48) continue;
                    std::vector<HWork> tmp;
                    nao_split_h_items(b, P, N, TN, S, tmp, F);
                    best_h = std::max(best_h, (int64_t)tmp.size());
                }
                cap_h += best_h;
                cap_n += G.n_qt;
            }
        }
        cur.b1 = c.b1;
        g->split_chunks.push_back(cur);
    }
    nao_status st;
    if ((st = dev_alloc(g, &g->d_slices, (size_t)std::max<int64_t>(max_used, 1024))) ||
        (st = upload(g, &g->d_sl_off_h, off_h.data(), off_h.size())) ||
        (st = upload(g, &g->d_sl_off_n, off_n.data(), off_n.size())) ||
        (st = dev_alloc(g, &g->d_expo_h, (size_t)std::max<int64_t>(g->rel_total, 1))) ||
        (st = dev_alloc(g, &g->d_expo_q, (size_t)g->n_points)) ||
        (st = dev_alloc(g, &g->d_expo_b, (size_t)g->n_batches)) ||
        (st = dev_alloc(g, &g->d_neg16, (size_t)g->n_batches)) ||
        (st = dev_alloc(g, &g->d_split_tn, (size_t)g->n_batches)) ||
        (st = dev_alloc(g, &g->d_split_hw, (size_t)std::max<int64_t>(cap_h, 1))) ||
        (st = dev_alloc(g, &g->d_split_nw, (size_t)std::max<int64_t>(cap_n, 1))))
        return st;
    g->cap_split_hw = cap_h;
    g->cap_split_nw = cap_n;
    g->split_S = S;
    g->split_F = F;
    g->split_tuned = nao_split_tn(S, F) != 48 || !g->opt.autotune;  // only one width exists, or tuning is off
    if ((st = split_lists(g))) return st;
    g->split_ready = true;
    return NAO_OK;
}

// Autotuner of the split path's tile width, driven by the batch-size histogram: batches are
// bucketed by (basis functions N_b, points P_b); for every bucket the H contraction of the
// bucket's batches in the first split chunks (repeated to fill the GPU for several waves, so
// that the timing is the throughput of a full launch) is timed with 128x48 and with 128x32
// tiles (CUDA events on the call's stream, the best of three runs after a warm-up, without the
// scatter), and
// 32 is kept for all batches of the bucket when it is at least 10 % faster (a second width
// costs a launch of its own; the density uses the same width). Buckets that
// none of those chunks contains keep the default rule. Runs once per handle, inside the first
// split Hamiltonian call (the evaluation and slicing it needs use that call's v and terms).
// N_b classes: steps of 16 up to 512 (the padding of the last 48- or 32-wide tile depends on N_b
// modulo the width), then steps of 128; P_b classes: 64, 128, 192, 256, 336, more.
constexpr int kTnBuckets = (32 + 5) * 6;
int tn_bucket(int N, int P) {
    static const int pe[] = {64, 128, 192, 256, 336};
    const int a = N <= 512 ? (N + 15) / 16 - 1 : (N <= 1024 ? 32 + (N - 513) / 128 : 36);
    int c = 0;
    while (c < 5 && P > pe[c]) c++;
    return a * 6 + c;
}

nao_status split_tune(nao_grid *g, uint32_t terms, cudaStream_t st) {
    if (g->split_tuned) return NAO_OK;
    const int S = g->split_S;
    const DevSystem &s = g->sys;
    constexpr int kBuckets = kTnBuckets, kChunks = 3;
    std::vector<int> bucket(g->n_batches, -1), total(kBuckets, 0);
    for (int64_t b = 0; b < g->n_batches; b++)
        if (g->Nb[b] > 0) {
            bucket[b] = tn_bucket(g->Nb[b], g->Pb[b]);
            total[bucket[b]]++;
        }
    std::vector<int> choice(kBuckets, 0);
    cudaEvent_t e0, e1;
    NAO_CUDA(cudaEventCreate(&e0));
    NAO_CUDA(cudaEventCreate(&e1));
    nao_status rs = NAO_OK;
    int timed = 0;
    for (size_t ci = 0; ci < g->split_chunks.size() && (int)ci < kChunks && rs == NAO_OK; ci++) {
        const auto &c = g->split_chunks[ci];
        bool any = false;
        for (int32_t b = c.b0; b < c.b1; b++) any = any || (bucket[b] >= 0 && !choice[bucket[b]]);
        if (!any) continue;
        cudaError_t ce = launch_eval(s, c.b0, c.b1, NAO_SPLIT, true, g->d_scratch, st);
        if (ce == cudaSuccess)
            ce = launch_slice_h(s, c.b0, c.b1, c.max_rt, g->d_scratch, terms, g->d_slices, g->d_sl_off_h, g->d_expo_h,
                                g->d_neg16, S, g->split_F, st);
        if (ce != cudaSuccess) { rs = cuda_fail(ce, "autotune evaluation"); break; }
        for (int k = 0; k < kBuckets && rs == NAO_OK; k++) {
            if (choice[k] || !total[k]) continue;
            float ms[2] = {0.0f, 0.0f};
            int64_t n_items = 0;
            // the bucket's batches of this chunk, repeated so that the 48-wide launch has at
            // least 8 CTAs per SM: the timing is throughput in a full launch, as in the real run
            int64_t base48 = 0;
            for (int32_t b = c.b0; b < c.b1; b++) {
                if (bucket[b] != k) continue;
                std::vector<HWork> tmp;
                nao_split_h_items(b, g->Pb[b], g->Nb[b], 48, S, tmp);
                base48 += (int64_t)tmp.size();
            }
            const int64_t reps = base48 > 0 ? (8 * 152 + base48 - 1) / base48 : 0;
            for (int w = 0; w < 2 && rs == NAO_OK && reps > 0; w++) {
                const int TN = w == 0 ? 48 : 32;
                std::vector<HWork> items;
                for (int64_t r = 0; r < reps; r++)
                    for (int32_t b = c.b0; b < c.b1; b++)
                        if (bucket[b] == k) nao_split_h_items(b, g->Pb[b], g->Nb[b], TN, S, items);
                n_items = (int64_t)items.size();
                if (items.empty()) break;
                if ((int64_t)items.size() > g->cap_tune_hw) {
                    if ((rs = dev_alloc(g, &g->d_tune_hw, items.size()))) break;
                    g->cap_tune_hw = (int64_t)items.size();
                }
                ce = copy_async(g->d_tune_hw, items.data(), items.size() * sizeof(HWork), cudaMemcpyHostToDevice,
                                     g->setup);
                if (ce == cudaSuccess) ce = cudaStreamSynchronize(g->setup);
                ms[w] = 1e30f;
                for (int rep = 0; rep < 4 && ce == cudaSuccess; rep++) {  // the first run warms up
                    ce = cudaEventRecord(e0, st);
                    if (ce == cudaSuccess)
                        ce = launch_h_tc(s, g->d_tune_hw, 0, (int32_t)items.size(), g->d_slices, g->d_sl_off_h,
                                         g->d_expo_h, g->d_neg16, S, g->split_F, TN, 0, g->d_err, st);
                    if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
                    if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
                    float t = 0.0f;
                    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
                    if (rep > 0) ms[w] = std::min(ms[w], t);
                }
                if (ce != cudaSuccess) rs = cuda_fail(ce, "autotune timing");
            }
            if (rs != NAO_OK || n_items == 0) continue;
            choice[k] = ms[1] < 0.9f * ms[0] ? 32 : 48;  // 32 only when clearly faster (it costs a launch)
            timed++;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != NAO_OK) return rs;
    for (int64_t b = 0; b < g->n_batches; b++)
        if (bucket[b] >= 0 && choice[bucket[b]]) g->split_tn[b] = choice[bucket[b]];
    g->tune_buckets = timed;
    g->split_tuned = true;
    return split_lists(g);
}

// This call's pointer tables (sections: 0 H, 1 v, 2 P, 3 n, 4 N_e; one entry per system),
// written on the call's stream by kernels that carry the values in their arguments.
nao_status upload_tables(nao_grid *g, int first, int count, cudaStream_t st) {
    const size_t n = (size_t)g->n_sys;
    if (fault_fires(FAULT_LAUNCH)) return cuda_fail(cudaErrorLaunchFailure, "launch_set_pointers");
    NAO_CUDA(launch_set_pointers(g->d_tab + first * n, g->h_tab.data() + first * n, (int32_t)(count * n), st));
    return NAO_OK;
}

// Runs enqueue(stream) either directly on st, or (capture_graph) as a CUDA graph replayed on
// the handle's own stream, ordered after st's prior work and before st's later work by events.
// The first call with a given key captures and instantiates the graph.
template <class F>
nao_status run_maybe_graph(nao_grid *g, uint64_t key, cudaStream_t st, F &&enqueue) {
    if (!g->opt.capture_graph || g->profiling) return enqueue(st);
    if (!g->gstream) {
        NAO_CUDA(cudaStreamCreateWithFlags(&g->gstream, cudaStreamNonBlocking));
        NAO_CUDA(cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming));
        NAO_CUDA(cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming));
    }
    NAO_CUDA(cudaEventRecord(g->ev_in, st));
    NAO_CUDA(cudaStreamWaitEvent(g->gstream, g->ev_in, 0));
    auto it = g->graphs.find(key);
    if (it == g->graphs.end()) {
        NAO_CUDA(cudaStreamBeginCapture(g->gstream, cudaStreamCaptureModeThreadLocal));
        const nao_status es = enqueue(g->gstream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(g->gstream, &graph);
        if (es != NAO_OK) {
            if (graph) cudaGraphDestroy(graph);
            return es;
        }
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) return cuda_fail(ie, "cudaGraphInstantiate");
        it = g->graphs.emplace(key, exec).first;
    }
    NAO_CUDA(cudaGraphLaunch(it->second, g->gstream));
    NAO_CUDA(cudaEventRecord(g->ev_out, g->gstream));
    NAO_CUDA(cudaStreamWaitEvent(st, g->ev_out, 0));
    return NAO_OK;
}

nao_status enqueue_h(nao_grid *g, uint32_t terms, nao_precision prec, cudaStream_t st) {
    const DevSystem &s = g->sys;
    NAO_CUDA(launch_zero_h(s, g->d_zero_tasks, (int32_t)g->zero_tasks.size(), st));
    if (prec == NAO_SPLIT) {
        const int S = g->split_S;
        for (const auto &c : g->split_chunks) {
            NAO_CUDA(timed(g, NAO_K_EVAL_GRAD, st, [&] { return launch_eval(s, c.b0, c.b1, NAO_SPLIT, true, g->d_scratch, st); }));
            NAO_CUDA(timed(g, NAO_K_SLICE, st, [&] {
                return launch_slice_h(s, c.b0, c.b1, c.max_rt, g->d_scratch, terms, g->d_slices, g->d_sl_off_h,
                                      g->d_expo_h, g->d_neg16, S, g->split_F, st);
            }));
            for (int k = 0; k < 2; k++)
                if (c.hw1[k] > c.hw0[k])
                NAO_CUDA(timed(g, NAO_K_H_SPLIT, st, [&] {
                    return launch_h_tc(s, g->d_split_hw, c.hw0[k], c.hw1[k] - c.hw0[k], g->d_slices, g->d_sl_off_h,
                                       g->d_expo_h, g->d_neg16, S, g->split_F, k == 0 ? 48 : 32, 1, g->d_err, st);
                }));
        }
    } else {
        for (const Chunk &c : g->chunks) {
            NAO_CUDA(timed(g, NAO_K_EVAL_GRAD, st, [&] { return launch_eval(s, c.b0, c.b1, prec, true, g->d_scratch, st); }));
            NAO_CUDA(timed(g, prec == NAO_FP32 ? NAO_K_H_FP32 : NAO_K_H_FP64, st, [&] {
                return launch_h_simt(s, prec, g->d_hwork + c.hw0, c.hw1 - c.hw0, g->d_scratch, terms, st);
            }));
        }
    }
    NAO_CUDA(timed(g, NAO_K_MIRROR, st, [&] { return launch_mirror(s, g->d_mirror_tasks, (int32_t)g->mirror_tasks.size(), st); }));
    return NAO_OK;
}

nao_status enqueue_n(nao_grid *g, nao_precision prec, bool want_ne, bool grad, cudaStream_t st) {
    const DevSystem &s = g->sys;
    if (prec == NAO_SPLIT) {
        const int S = g->split_S;
        NAO_CUDA(launch_zero_n(s, g->d_dwork, (int32_t)g->n_dwork, grad, st));
        for (const auto &c : g->split_chunks) {
            NAO_CUDA(timed(g, grad ? NAO_K_EVAL_GRAD : NAO_K_EVAL_PHI, st, [&] {
                return launch_eval_split(s, c.b0, c.b1, grad, g->d_scratch, g->d_expo_q, 128 * c.max_qt, st);
            }));
            NAO_CUDA(timed(g, NAO_K_SLICE_N, st, [&] {
                return launch_slice_n(s, c.b0, c.b1, c.max_qt, c.max_rt, g->d_scratch, g->d_slices, g->d_sl_off_n,
                                      g->d_expo_q, g->d_expo_b, g->d_split_tn, S, g->split_F, grad, st);
            }));
            for (int k = 0; k < 2; k++)
                if (c.nw1[k] > c.nw0[k])
                NAO_CUDA(timed(g, NAO_K_N_SPLIT, st, [&] {
                    return launch_n_tc(s, g->d_split_nw, c.nw0[k], c.nw1[k] - c.nw0[k], g->d_slices, g->d_sl_off_n,
                                       g->d_expo_q, g->d_expo_b, g->d_scratch, S, g->split_F, k == 0 ? 48 : 32, grad, g->d_err,
                                       st);
                }));
        }
        if (want_ne) NAO_CUDA(launch_wn_partial(s, g->d_dwork, 0, (int32_t)g->n_dwork, g->d_ne_part, st));
    } else {
        for (const Chunk &c : g->chunks) {
            NAO_CUDA(timed(g, grad ? NAO_K_EVAL_GRAD : NAO_K_EVAL_PHI, st,
                           [&] { return launch_eval(s, c.b0, c.b1, prec, grad, g->d_scratch, st); }));
            NAO_CUDA(timed(g, prec == NAO_FP32 ? NAO_K_N_FP32 : NAO_K_N_FP64, st, [&] {
                return launch_density_simt(s, prec, g->d_dwork, c.dw0, c.dw1 - c.dw0, g->d_scratch, g->d_ne_part, grad,
                                           st);
            }));
        }
    }
    if (want_ne)
        NAO_CUDA(timed(g, NAO_K_REDUCE, st, [&] { return launch_reduce_ne(s, g->d_ne_part, g->d_sys_dw0, g->n_sys, st); }));
    return NAO_OK;
}

// H of every system from the tables' sections 0 (H) and 1 (v), already filled in g->h_tab.
nao_status run_h(nao_grid *g, uint32_t terms, nao_precision prec, cudaStream_t st) {
    nao_status rs;
    if (prec == NAO_SPLIT && (rs = split_setup(g))) return rs;
    if ((rs = upload_tables(g, 0, 2, st))) return rs;
    if ((terms & NAO_TERM_TAU) && (rs = upload_tables(g, 6, 1, st))) return rs;
    if (prec == NAO_SPLIT && (rs = split_tune(g, terms, st))) return rs;
    const uint64_t key = (uint64_t)1 << 40 | (uint64_t)prec << 8 | terms;
    return run_maybe_graph(g, key, st, [&](cudaStream_t s2) { return enqueue_h(g, terms, prec, s2); });
}

// n (and N_e where a table entry is set, grad n when asked for) of every system from sections
// 2 (P), 3 (n), 4 (N_e), 5 (grad n).
nao_status run_n(nao_grid *g, nao_precision prec, cudaStream_t st, bool grad = false) {
    nao_status rs;
    if (prec == NAO_SPLIT && (rs = split_setup(g))) return rs;
    if ((rs = upload_tables(g, 2, grad ? 4 : 3, st))) return rs;
    bool want_ne = false;
    for (int m = 0; m < g->n_sys; m++) want_ne = want_ne || g->h_tab[4 * (size_t)g->n_sys + m] != nullptr;
    const uint64_t key = (uint64_t)2 << 40 | (uint64_t)prec << 8 | (want_ne ? 1u : 0u) | (grad ? 2u : 0u);
    return run_maybe_graph(g, key, st, [&](cudaStream_t s2) { return enqueue_n(g, prec, want_ne, grad, s2); });
}

void set_tab(nao_grid *g, int section, int m, const void *p) { g->h_tab[(size_t)section * g->n_sys + m] = const_cast<void *>(p); }

// Density Hessian plan: runs of batches whose evaluation in the 10-row layout (phi, grad phi,
// six second derivatives: N_b x 10 Ppad FP64 per batch) fits the evaluation scratch, their
// density work items (64-point tiles, consecutive per batch) and the per-batch offsets.
nao_status hess_plan(nao_grid *g) {
    if (!g->hess_chunks.empty()) return NAO_OK;
    const int64_t nbat = g->n_batches;
    std::vector<int64_t> off((size_t)std::max<int64_t>(nbat, 1), 0);
    int64_t used = 0, dw = 0;
    nao_grid::HessChunk cur{0, 0, 0, 0};
    for (int64_t b = 0; b < nbat; b++) {
        const int64_t Ppad = (g->Pb[b] + NAO_PPAD - 1) / NAO_PPAD * NAO_PPAD;
        const int64_t e = (int64_t)g->Nb[b] * 10 * Ppad;
        if (e > g->scratch_elems)
            return fail(NAO_ERR_UNSUPPORTED, "density Hessian: batch " + std::to_string(b) +
                                                 " needs more evaluation scratch than the handle has (raise scratch_bytes)");
        if (used + e > g->scratch_elems && b > cur.b0) {
            cur.b1 = (int32_t)b;
            cur.dw1 = (int32_t)dw;
            g->hess_chunks.push_back(cur);
            cur = nao_grid::HessChunk{(int32_t)b, 0, (int32_t)dw, 0};
            used = 0;
        }
        off[(size_t)b] = used;
        used += e;
        dw += (g->Pb[b] + NAO_TILE - 1) / NAO_TILE;
    }
    cur.b1 = (int32_t)nbat;
    cur.dw1 = (int32_t)dw;
    g->hess_chunks.push_back(cur);
    if (dw != g->n_dwork) {
        g->hess_chunks.clear();
        return fail(NAO_ERR_INTERNAL, "density Hessian: work items do not match the density tiles");
    }
    nao_status st = upload(g, &g->d_hess_off, off.data(), off.size());
    if (st) {
        g->hess_chunks.clear();
        return st;
    }
    NAO_CUDA(cudaStreamSynchronize(g->setup));
    return NAO_OK;
}

// Local Pulay terms plan (after hess_plan): every 64 x 64 tile pair of every batch, in the order of
// the Hessian chunks, and the atoms' basis offsets on the device.
nao_status pulay_plan(nao_grid *g) {
    if (g->d_pulay_work) return NAO_OK;
    nao_status st;
    if ((st = hess_plan(g))) return st;
    std::vector<HWork> items;
    g->pulay_w0.assign(1, 0);
    for (const auto &c : g->hess_chunks) {
        for (int32_t b = c.b0; b < c.b1; b++) {
            const int nt = (g->Nb[b] + NAO_TILE - 1) / NAO_TILE;
            for (int I = 0; I < nt; I++)
                for (int J = 0; J < nt; J++) items.push_back({b, I, J, 0});
        }
        g->pulay_w0.push_back((int32_t)items.size());
    }
    if (items.empty()) items.push_back({0, 0, 0, 0});  // keeps the device array non-empty
    if ((st = upload(g, &g->d_pulay_work, items.data(), items.size())) ||
        (st = upload(g, &g->d_atom_basis, g->atom_basis.data(), g->atom_basis.size()))) {
        g->d_pulay_work = nullptr;
        return st;
    }
    NAO_CUDA(cudaStreamSynchronize(g->setup));
    return NAO_OK;
}

}  // namespace

void nao_set_last_error(const std::string &msg) { g_last_error = msg; }

extern "C" {

nao_status nao_default_options(nao_options *o) {
    if (!o) return fail(NAO_ERR_INVALID_ARG, "opts is NULL");
    std::memset(o, 0, sizeof(*o));
    o->max_batch_points = 200;
    o->split_slices = 12;
    o->deterministic = 0;
    o->device = -1;
    o->scratch_bytes = 0;
    o->capture_graph = 0;
    o->autotune = 1;
    o->split_digits = NAO_DIGITS_BF16;
    return NAO_OK;
}

static nao_status create(const nao_system_desc *descs, int32_t n_sys, const int32_t *batch_points,
                         const nao_options *opts, nao_grid **out) {
    if (!out) return fail(NAO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!descs) return fail(NAO_ERR_INVALID_ARG, "desc is NULL");
    if (n_sys < 1) return fail(NAO_ERR_INVALID_ARG, "n_systems < 1");
    nao_options o;
    nao_default_options(&o);
    if (opts) o = *opts;
    if (o.autotune != 0 && o.autotune != 1) return fail(NAO_ERR_INVALID_ARG, "options.autotune not 0/1");
    if (o.capture_graph != 0 && o.capture_graph != 1) return fail(NAO_ERR_INVALID_ARG, "options.capture_graph not 0/1");
    if (o.deterministic != 0 && o.deterministic != 1) return fail(NAO_ERR_INVALID_ARG, "options.deterministic not 0/1");
    nao_status st;
    if (batch_points)
        for (int32_t m = 0; m < n_sys; m++)
            if (batch_points[m] < 1 || batch_points[m] > NAO_MAX_BATCH)
                return fail(NAO_ERR_INVALID_ARG, "max_batch_points[" + std::to_string(m) + "] outside 1.." +
                                                     std::to_string(NAO_MAX_BATCH));
    for (int32_t m = 0; m < n_sys; m++)
        if ((st = validate(&descs[m], o)) != NAO_OK) {
            if (n_sys > 1) g_last_error = "system " + std::to_string(m) + ": " + g_last_error;
            return st;
        }
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(NAO_ERR_CUDA, "no CUDA device");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || dev >= ndev) {
        cudaGetLastError();
        return fail(NAO_ERR_INVALID_ARG, "bad device ordinal");
    }
    DeviceGuard guard(dev);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    // Per-thread stack of this process's context: the evaluation kernels' frames (their per-l
    // evaluation functions are calls, not inlined) reach about 1 KB, the default limit; the
    // limit is raised to kStackBytes if it is lower (a limit of this context only, which ends
    // with the process).
    {
        constexpr size_t kStackBytes = 2048;
        size_t cur = 0;
        if (cudaDeviceGetLimit(&cur, cudaLimitStackSize) != cudaSuccess ||
            (cur < kStackBytes && cudaDeviceSetLimit(cudaLimitStackSize, kStackBytes) != cudaSuccess)) {
            cudaGetLastError();
            return fail(NAO_ERR_CUDA, "cannot set the per-thread stack size");
        }
    }
    nao_grid *g = new (std::nothrow) nao_grid();
    if (!g) return fail(NAO_ERR_OUT_OF_MEMORY, "host allocation failed");
    g->device = dev;
    g->opt = o;
    g->opt.device = dev;
    try {
        st = init_streams(g);
        if (st == NAO_OK) st = build(g, descs, n_sys, batch_points);
    } catch (const std::bad_alloc &) {
        st = fail(NAO_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        st = fail(NAO_ERR_INTERNAL, "unexpected host exception");
    }
    if (st != NAO_OK) {
        free_grid(g);
        return st;
    }
    *out = g;
    return NAO_OK;
}

nao_status nao_grid_create(const nao_system_desc *desc, const nao_options *opts, nao_grid **out) {
    return create(desc, 1, nullptr, opts, out);
}

nao_status nao_grid_create_many(const nao_system_desc *descs, int32_t n_systems, const int32_t *max_batch_points,
                                const nao_options *opts, nao_grid **out) {
    return create(descs, n_systems, max_batch_points, opts, out);
}

nao_status nao_get_system(const nao_grid *g, int32_t m, int64_t *basis_offset, int64_t *n_basis, int64_t *point_offset,
                          int64_t *n_points, int64_t *batch_begin, int64_t *batch_end) {
    nao_status st = check_handle(g);
    if (st) return st;
    if (m < 0 || m >= g->n_sys) return fail(NAO_ERR_INVALID_ARG, "system index out of range");
    if (basis_offset) *basis_offset = g->sys_boff[m];
    if (n_basis) *n_basis = g->sys_nb[m];
    if (point_offset) *point_offset = g->sys_poff[m];
    if (n_points) *n_points = g->sys_np[m];
    if (batch_begin || batch_end) {
        // batches of system m are contiguous; their points are the system's point range
        const int64_t p0 = g->sys_poff[m], p1 = p0 + g->sys_np[m];
        const auto b0 = std::lower_bound(g->batch_off.begin(), g->batch_off.end(), p0) - g->batch_off.begin();
        const auto b1 = std::lower_bound(g->batch_off.begin(), g->batch_off.end(), p1) - g->batch_off.begin();
        if (batch_begin) *batch_begin = b0;
        if (batch_end) *batch_end = b1;
    }
    return NAO_OK;
}

nao_status nao_destroy(nao_grid *g) {
    if (!g) return NAO_OK;
    DeviceGuard guard(g->device);
    free_grid(g);
    return NAO_OK;
}

nao_status nao_get_info(const nao_grid *g, nao_grid_info *info) {
    nao_status st = check_handle(g);
    if (st) return st;
    if (!info) return fail(NAO_ERR_INVALID_ARG, "info is NULL");
    info->n_basis = g->nb;
    info->n_points = g->n_points;
    info->n_batches = g->n_batches;
    info->rel_total = g->rel_total;
    info->max_batch_points = g->max_P;
    info->max_batch_basis = g->max_N;
    info->device_bytes = g->dev_bytes;
    info->flops_h = g->flops_h;
    info->flops_n = g->flops_n;
    info->n_systems = g->n_sys;
    info->n_atoms = g->n_atoms;
    return NAO_OK;
}

nao_status nao_export_batches(const nao_grid *g, int64_t *batch_offsets, int64_t *point_perm, int64_t *rel_offsets,
                              int32_t *rel_idx) {
    nao_status st = check_handle(g);
    if (st) return st;
    if (batch_offsets) std::memcpy(batch_offsets, g->batch_off.data(), g->batch_off.size() * sizeof(int64_t));
    if (point_perm) std::memcpy(point_perm, g->perm.data(), g->perm.size() * sizeof(int64_t));
    if (rel_offsets) std::memcpy(rel_offsets, g->rel_off.data(), g->rel_off.size() * sizeof(int64_t));
    if (rel_idx && g->rel_total) std::memcpy(rel_idx, g->rel_idx.data(), g->rel_idx.size() * sizeof(int32_t));
    return NAO_OK;
}

nao_status nao_partition_points(const double *pt_xyz, int64_t n_points, int64_t max_batch_points, int64_t max_batches,
                                int64_t *batch_offsets, int64_t *point_perm, int64_t *n_batches) {
    if (!pt_xyz || !n_batches || n_points < 1 || max_batch_points < 1 || max_batches < 0)
        return fail(NAO_ERR_INVALID_ARG, "nao_partition_points: bad argument");
    for (int64_t k = 0; k < 3 * n_points; k++)
        if (!std::isfinite(pt_xyz[k])) return fail(NAO_ERR_INVALID_ARG, "nao_partition_points: non-finite coordinate");
    std::vector<int64_t> off, perm;
    try {
        *n_batches = nao_partition(n_points, pt_xyz, max_batch_points, off, perm);
    } catch (const std::bad_alloc &) {
        return fail(NAO_ERR_OUT_OF_MEMORY, "nao_partition_points: host memory");
    }
    if (*n_batches > max_batches)
        return fail(NAO_ERR_INVALID_ARG, "nao_partition_points: " + std::to_string(*n_batches) +
                                             " batches exceed max_batches (n_batches holds the count)");
    if (!batch_offsets || !point_perm) return fail(NAO_ERR_INVALID_ARG, "nao_partition_points: NULL output");
    std::memcpy(batch_offsets, off.data(), off.size() * sizeof(int64_t));
    std::memcpy(point_perm, perm.data(), perm.size() * sizeof(int64_t));
    return NAO_OK;
}

nao_status nao_radial_spline(const double *fn_table, int32_t n_rgrid, double *coef) {
    if (!fn_table || !coef || n_rgrid < 4) return fail(NAO_ERR_INVALID_ARG, "nao_radial_spline: bad argument");
    for (int32_t k = 0; k < n_rgrid; k++)
        if (!std::isfinite(fn_table[k])) return fail(NAO_ERR_INVALID_ARG, "nao_radial_spline: non-finite table entry");
    nao_spline_coefficients(fn_table, n_rgrid, coef);
    return NAO_OK;
}

static nao_status check_single(const nao_grid *g) {
    if (g->n_sys != 1)
        return fail(NAO_ERR_INVALID_ARG,
                    "the handle holds " + std::to_string(g->n_sys) + " systems; use the _many entry points");
    return NAO_OK;
}

static nao_status check_terms(uint32_t terms) {
    if (terms == 0 || (terms & ~3u)) return fail(NAO_ERR_INVALID_ARG, "bad terms");
    return NAO_OK;
}

nao_status nao_get_tuning(const nao_grid *g, int32_t *tile_width, int32_t *buckets_timed) {
    nao_status st = check_handle(g);
    if (st) return st;
    if (tile_width) {
        if (g->split_ready) std::memcpy(tile_width, g->split_tn.data(), g->split_tn.size() * sizeof(int32_t));
        else std::memset(tile_width, 0, (size_t)g->n_batches * sizeof(int32_t));
    }
    if (buckets_timed) *buckets_timed = g->split_tuned ? g->tune_buckets : -1;
    return NAO_OK;
}

nao_status nao_integrate_h(nao_grid *g, const double *v_dev, uint32_t terms, nao_precision prec, double *H_dev,
                           void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st || (st = check_single(g))) return st;
    if (!H_dev) return fail(NAO_ERR_INVALID_ARG, "H_dev is NULL");
    if ((st = check_terms(terms)) || (st = check_prec(prec))) return st;
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    set_tab(g, 0, 0, H_dev);
    set_tab(g, 1, 0, v_dev);
    if ((st = run_h(g, terms, prec, static_cast<cudaStream_t>(cuda_stream)))) return st;
    return mark_done(g, static_cast<cudaStream_t>(cuda_stream));
}
nao_status nao_integrate_h_tau(nao_grid *g, const double *v_dev, const double *vtau_dev, uint32_t terms,
                               nao_precision prec, double *H_dev, void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st || (st = check_single(g))) return st;
    if (!H_dev) return fail(NAO_ERR_INVALID_ARG, "H_dev is NULL");
    if (terms == 0 || (terms & ~7u)) return fail(NAO_ERR_INVALID_ARG, "bad terms");
    if ((terms & NAO_TERM_TAU) && !vtau_dev) return fail(NAO_ERR_INVALID_ARG, "NAO_TERM_TAU needs vtau_dev");
    if ((st = check_prec(prec))) return st;
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    set_tab(g, 0, 0, H_dev);
    set_tab(g, 1, 0, v_dev);
    set_tab(g, 6, 0, (terms & NAO_TERM_TAU) ? vtau_dev : nullptr);
    if ((st = run_h(g, terms, prec, static_cast<cudaStream_t>(cuda_stream)))) return st;
    return mark_done(g, static_cast<cudaStream_t>(cuda_stream));
}


nao_status nao_integrate_h_many(nao_grid *g, const double *const *v_dev, uint32_t terms, nao_precision prec,
                                double *const *H_dev, void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st) return st;
    if (!H_dev) return fail(NAO_ERR_INVALID_ARG, "H_dev is NULL");
    for (int m = 0; m < g->n_sys; m++)
        if (!H_dev[m]) return fail(NAO_ERR_INVALID_ARG, "H_dev[" + std::to_string(m) + "] is NULL");
    if ((st = check_terms(terms)) || (st = check_prec(prec))) return st;
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    for (int m = 0; m < g->n_sys; m++) {
        set_tab(g, 0, m, H_dev[m]);
        set_tab(g, 1, m, v_dev ? v_dev[m] : nullptr);
    }
    if ((st = run_h(g, terms, prec, static_cast<cudaStream_t>(cuda_stream)))) return st;
    return mark_done(g, static_cast<cudaStream_t>(cuda_stream));
}

nao_status nao_update_density(nao_grid *g, const double *P_dev, nao_precision prec, double *n_dev,
                              double *n_electrons_dev, void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st || (st = check_single(g))) return st;
    if (!P_dev || !n_dev) return fail(NAO_ERR_INVALID_ARG, "P_dev or n_dev is NULL");
    if ((st = check_prec(prec))) return st;
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    set_tab(g, 2, 0, P_dev);
    set_tab(g, 3, 0, n_dev);
    set_tab(g, 4, 0, n_electrons_dev);
    if ((st = run_n(g, prec, static_cast<cudaStream_t>(cuda_stream)))) return st;
    return mark_done(g, static_cast<cudaStream_t>(cuda_stream));
}

nao_status nao_update_density_many(nao_grid *g, const double *const *P_dev, nao_precision prec, double *const *n_dev,
                                   double *const *n_electrons_dev, void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st) return st;
    if (!P_dev || !n_dev) return fail(NAO_ERR_INVALID_ARG, "P_dev or n_dev is NULL");
    for (int m = 0; m < g->n_sys; m++)
        if (!P_dev[m] || !n_dev[m])
            return fail(NAO_ERR_INVALID_ARG, "P_dev[" + std::to_string(m) + "] or n_dev[" + std::to_string(m) + "] is NULL");
    if ((st = check_prec(prec))) return st;
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    for (int m = 0; m < g->n_sys; m++) {
        set_tab(g, 2, m, P_dev[m]);
        set_tab(g, 3, m, n_dev[m]);
        set_tab(g, 4, m, n_electrons_dev ? n_electrons_dev[m] : nullptr);
    }
    if ((st = run_n(g, prec, static_cast<cudaStream_t>(cuda_stream)))) return st;
    return mark_done(g, static_cast<cudaStream_t>(cuda_stream));
}

nao_status nao_update_density_gradient_many(nao_grid *g, const double *const *P_dev, nao_precision prec,
                                            double *const *n_dev, double *const *grad_dev,
                                            double *const *n_electrons_dev, void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st) return st;
    if (!P_dev || !n_dev || !grad_dev) return fail(NAO_ERR_INVALID_ARG, "P_dev, n_dev or grad_dev is NULL");
    for (int m = 0; m < g->n_sys; m++)
        if (!P_dev[m] || !n_dev[m] || !grad_dev[m])
            return fail(NAO_ERR_INVALID_ARG, "P_dev, n_dev or grad_dev entry " + std::to_string(m) + " is NULL");
    if ((st = check_prec(prec))) return st;
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    for (int m = 0; m < g->n_sys; m++) {
        set_tab(g, 2, m, P_dev[m]);
        set_tab(g, 3, m, n_dev[m]);
        set_tab(g, 4, m, n_electrons_dev ? n_electrons_dev[m] : nullptr);
        set_tab(g, 5, m, grad_dev[m]);
    }
    if ((st = run_n(g, prec, static_cast<cudaStream_t>(cuda_stream), true))) return st;
    return mark_done(g, static_cast<cudaStream_t>(cuda_stream));
}

nao_status nao_update_density_gradient(nao_grid *g, const double *P_dev, nao_precision prec, double *n_dev,
                                       double *grad_dev, double *n_electrons_dev, void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st || (st = check_single(g))) return st;
    double *const ne[1] = {n_electrons_dev};
    return nao_update_density_gradient_many(g, &P_dev, prec, &n_dev, &grad_dev, ne, cuda_stream);
}

// Split-path density Hessian plan (after split_setup and hess_plan): every non-empty
// intersection of a Hessian chunk (the 10-row FP64 evaluation) with a split chunk (the slices),
// its slicing grid extents and its density work items (all function tiles per 128-point tile,
// heaviest first, per tile width), and the four point-exponent arrays.
nao_status hess_split_plan(nao_grid *g) {
    if (g->hess_split_ver == g->split_lists_ver && !g->hess_split.empty()) return NAO_OK;
    const int S = g->split_S, F = g->split_F;
    g->hess_split.clear();
    std::vector<HWork> nw[2];
    for (const auto &hc : g->hess_chunks)
        for (const auto &sc : g->split_chunks) {
            const int32_t lo = std::max(hc.b0, sc.b0), hi = std::min(hc.b1, sc.b1);
            if (lo >= hi) continue;
            nao_grid::HessSplitSub sub{lo, hi, 0, 0, {0, 0}, {0, 0}};
            for (int k = 0; k < 2; k++) sub.nw0[k] = (int32_t)nw[k].size();
            for (int32_t b = lo; b < hi; b++) {
                const int P = g->Pb[b], N = g->Nb[b];
                if (N == 0) continue;
                const int TN = g->split_tn[b], k = TN == 48 ? 0 : 1;
                const SplitGeom G(P, N, S, TN, F);
                sub.max_qt = std::max<int32_t>(sub.max_qt, G.n_qt);
                sub.max_rt = std::max<int32_t>(sub.max_rt, G.h_slice_tiles());
                for (int Q = 0; Q < G.n_qt; Q++) nw[k].push_back({b, Q, G.n_jtN, 0});
            }
            for (int k = 0; k < 2; k++) {
                std::stable_sort(nw[k].begin() + sub.nw0[k], nw[k].end(),
                                 [](const HWork &x, const HWork &y) { return x.tj > y.tj; });
                sub.nw1[k] = (int32_t)nw[k].size();
            }
            g->hess_split.push_back(sub);
        }
    for (auto &sub : g->hess_split) {
        sub.nw0[1] += (int32_t)nw[0].size();
        sub.nw1[1] += (int32_t)nw[0].size();
    }
    nw[0].insert(nw[0].end(), nw[1].begin(), nw[1].end());
    nao_status st;
    if ((int64_t)nw[0].size() > g->cap_hess_nw) {
        if (g->d_hess_nw) {
            NAO_CUDA(cudaStreamSynchronize(g->setup));
            g->d_hess_nw = nullptr;  // the old list stays in g->allocs until the handle is destroyed
        }
        if ((st = dev_alloc(g, &g->d_hess_nw, std::max<size_t>(nw[0].size(), 1)))) {
            g->hess_split.clear();
            return st;
        }
        g->cap_hess_nw = (int64_t)std::max<size_t>(nw[0].size(), 1);
    }
    if (!g->d_expo4 && (st = dev_alloc(g, &g->d_expo4, 4 * (size_t)std::max<int64_t>(g->n_points, 1)))) {
        g->hess_split.clear();
        return st;
    }
    if (!nw[0].empty())
        NAO_CUDA(copy_async(g->d_hess_nw, nw[0].data(), nw[0].size() * sizeof(HWork), cudaMemcpyHostToDevice, g->setup));
    NAO_CUDA(cudaStreamSynchronize(g->setup));
    g->hess_split_ver = g->split_lists_ver;
    return NAO_OK;
}

nao_status nao_update_density_hessian(nao_grid *g, const double *P_dev, nao_precision prec, double *n_dev,
                                      double *grad_dev, double *hess_dev, double *n_electrons_dev, void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st || (st = check_single(g))) return st;
    if (!P_dev || !n_dev || !grad_dev || !hess_dev)
        return fail(NAO_ERR_INVALID_ARG, "P_dev, n_dev, grad_dev or hess_dev is NULL");
    if ((st = check_prec(prec))) return st;
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    if (prec == NAO_SPLIT && (st = split_setup(g))) return st;
    if ((st = hess_plan(g))) return st;
    if (prec == NAO_SPLIT && (st = hess_split_plan(g))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    set_tab(g, 2, 0, P_dev);
    set_tab(g, 3, 0, n_dev);
    set_tab(g, 4, 0, n_electrons_dev);
    set_tab(g, 5, 0, grad_dev);
    if ((st = upload_tables(g, 2, 4, s))) return st;
    const DevSystem &sys = g->sys;
    if (prec == NAO_SPLIT) {
        // points of batches without basis functions get zeros; every other point is written by
        // the first pass and completed by the three later ones
        NAO_CUDA(cudaMemsetAsync(hess_dev, 0, 6 * (size_t)g->n_points * sizeof(double), s));
        NAO_CUDA(launch_zero_n(sys, g->d_dwork, (int32_t)g->n_dwork, true, s));
        const int S = g->split_S, F = g->split_F;
        size_t k_sub = 0;
        for (const auto &c : g->hess_chunks) {
            NAO_CUDA(launch_eval_hess(sys, c.b0, c.b1, g->d_scratch, false, false, g->d_hess_off, s));
            NAO_CUDA(launch_hess_point_expo(sys, c.b0, c.b1, g->d_scratch, g->d_hess_off, g->d_expo4, g->n_points, s));
            for (; k_sub < g->hess_split.size() && g->hess_split[k_sub].b0 < c.b1; k_sub++) {
                const auto &sub = g->hess_split[k_sub];
                for (int comp = 0; comp < 4; comp++) {
                    const int32_t *eq = g->d_expo4 + (size_t)comp * (size_t)g->n_points;
                    NAO_CUDA(launch_slice_n_hess(sys, sub.b0, sub.b1, sub.max_qt, sub.max_rt, g->d_scratch,
                                                 g->d_hess_off, comp, g->d_slices, g->d_sl_off_n, eq, g->d_expo_b,
                                                 g->d_split_tn, S, F, s));
                    for (int k = 0; k < 2; k++)
                        NAO_CUDA(launch_n_tc_hess(sys, g->d_hess_nw, sub.nw0[k], sub.nw1[k] - sub.nw0[k], g->d_slices,
                                                  g->d_sl_off_n, eq, g->d_expo_b, g->d_scratch, g->d_hess_off, comp,
                                                  hess_dev, S, F, k == 0 ? 48 : 32, g->d_err, s));
                }
            }
        }
        if (n_electrons_dev) {
            NAO_CUDA(launch_wn_partial(sys, g->d_dwork, 0, (int32_t)g->n_dwork, g->d_ne_part, s));
            NAO_CUDA(launch_reduce_ne(sys, g->d_ne_part, g->d_sys_dw0, g->n_sys, s));
        }
        return mark_done(g, s);
    }
    for (const auto &c : g->hess_chunks) {
        NAO_CUDA(launch_eval_hess(sys, c.b0, c.b1, g->d_scratch, prec == NAO_FP32, false, g->d_hess_off, s));
        NAO_CUDA(launch_density_hess(sys, g->d_dwork, c.dw0, c.dw1 - c.dw0, g->d_scratch, prec == NAO_FP32,
                                     g->d_hess_off, hess_dev, g->d_ne_part, s));
    }
    if (n_electrons_dev) NAO_CUDA(launch_reduce_ne(sys, g->d_ne_part, g->d_sys_dw0, g->n_sys, s));
    return mark_done(g, s);
}

nao_status nao_pulay_matrices(nao_grid *g, const double *v_dev, nao_precision prec, double *M_dev, double *S_dev,
                              void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st || (st = check_single(g))) return st;
    if (!M_dev || !S_dev) return fail(NAO_ERR_INVALID_ARG, "M_dev or S_dev is NULL");
    if ((st = check_prec(prec))) return st;
    if (prec == NAO_SPLIT)
        return fail(NAO_ERR_UNSUPPORTED, "the Pulay matrix elements are built on the FP64 and FP32 paths only");
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    if ((st = pulay_plan(g))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    set_tab(g, 1, 0, v_dev);
    if ((st = upload_tables(g, 1, 1, s))) return st;
    const size_t bytes = 3 * (size_t)g->nb * (size_t)g->nb * sizeof(double);
    NAO_CUDA(cudaMemsetAsync(M_dev, 0, bytes, s));
    NAO_CUDA(cudaMemsetAsync(S_dev, 0, bytes, s));
    const DevSystem &sys = g->sys;
    for (size_t k = 0; k < g->hess_chunks.size(); k++) {
        const auto &c = g->hess_chunks[k];
        NAO_CUDA(launch_eval_hess(sys, c.b0, c.b1, g->d_scratch, prec == NAO_FP32, true, g->d_hess_off, s));
        NAO_CUDA(launch_pulay(sys, g->d_pulay_work, g->pulay_w0[k], g->pulay_w0[k + 1] - g->pulay_w0[k], g->d_scratch,
                              prec == NAO_FP32, g->d_hess_off, M_dev, S_dev, g->nb, s));
    }
    return mark_done(g, s);
}

nao_status nao_pulay_forces(nao_grid *g, const double *n_dev, const double *q_dev, const double *M_dev,
                            const double *S_dev, double *F_dev, void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st || (st = check_single(g))) return st;
    if (!n_dev || !q_dev || !M_dev || !S_dev || !F_dev) return fail(NAO_ERR_INVALID_ARG, "a buffer is NULL");
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    if ((st = pulay_plan(g))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    NAO_CUDA(launch_pulay_forces(n_dev, q_dev, M_dev, S_dev, g->d_atom_basis, g->n_atoms, g->nb, F_dev, s));
    return mark_done(g, s);
}

static nao_status ensure_staging(nao_grid *g) {
    if (g->d_stage_in && g->d_stage_out && g->d_stage_ne) return NAO_OK;
    const size_t big = (size_t)std::max<int64_t>(g->nb * g->nb, g->n_points);
    nao_status st;
    if ((st = dev_alloc(g, &g->d_stage_in, big)) || (st = dev_alloc(g, &g->d_stage_out, big)) ||
        (st = dev_alloc(g, &g->d_stage_ne, 1)))
        return st;
    NAO_CUDA(cudaStreamSynchronize(g->setup));
    return NAO_OK;
}

nao_status nao_integrate_h_host(nao_grid *g, const double *v_host, uint32_t terms, nao_precision prec, double *H_host,
                                void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st || (st = check_single(g))) return st;
    if (!H_host) return fail(NAO_ERR_INVALID_ARG, "H_host is NULL");
    if ((st = check_terms(terms)) || (st = check_prec(prec))) return st;
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    if ((st = ensure_staging(g))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const double *v = nullptr;
    if (v_host) {
        NAO_CUDA(copy_async(g->d_stage_in, v_host, (size_t)g->n_points * sizeof(double), cudaMemcpyHostToDevice, s));
        v = g->d_stage_in;
    }
    set_tab(g, 0, 0, g->d_stage_out);
    set_tab(g, 1, 0, v);
    if ((st = run_h(g, terms, prec, s))) return st;
    NAO_CUDA(copy_async(H_host, g->d_stage_out, (size_t)g->nb * g->nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    if ((st = mark_done(g, s))) return st;
    NAO_CUDA(cudaStreamSynchronize(s));
    return NAO_OK;
}

nao_status nao_update_density_host(nao_grid *g, const double *P_host, nao_precision prec, double *n_host,
                                   double *n_electrons_host, void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st || (st = check_single(g))) return st;
    if (!P_host || !n_host) return fail(NAO_ERR_INVALID_ARG, "P_host or n_host is NULL");
    if ((st = check_prec(prec))) return st;
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    if ((st = ensure_staging(g))) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    NAO_CUDA(copy_async(g->d_stage_in, P_host, (size_t)g->nb * g->nb * sizeof(double), cudaMemcpyHostToDevice, s));
    set_tab(g, 2, 0, g->d_stage_in);
    set_tab(g, 3, 0, g->d_stage_out);
    set_tab(g, 4, 0, n_electrons_host ? g->d_stage_ne : nullptr);
    if ((st = run_n(g, prec, s))) return st;
    NAO_CUDA(copy_async(n_host, g->d_stage_out, (size_t)g->n_points * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (n_electrons_host)
        NAO_CUDA(copy_async(n_electrons_host, g->d_stage_ne, sizeof(double), cudaMemcpyDeviceToHost, s));
    if ((st = mark_done(g, s))) return st;
    NAO_CUDA(cudaStreamSynchronize(s));
    return NAO_OK;
}

nao_status nao_evaluate_batch(nao_grid *g, int64_t batch, nao_precision prec, double *phi_dev, double *grad_dev,
                              void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st) return st;
    if (batch < 0 || batch >= g->n_batches) return fail(NAO_ERR_INVALID_ARG, "batch out of range");
    if (g->Nb[batch] == 0) return NAO_OK;  // nothing to write
    if (!phi_dev) return fail(NAO_ERR_INVALID_ARG, "phi_dev is NULL");
    if ((st = check_prec(prec))) return st;
    DeviceGuard guard(g->device);
    if (!guard.ok) return fail(NAO_ERR_CUDA, "cannot select the device");
    CallEnd call_end(g, static_cast<cudaStream_t>(cuda_stream));
    NAO_CUDA(launch_eval_one(g->sys, (int32_t)batch, prec, phi_dev, grad_dev, static_cast<cudaStream_t>(cuda_stream)));
    return mark_done(g, static_cast<cudaStream_t>(cuda_stream));
}

nao_status nao_profile_enable(nao_grid *g, int32_t enable) {
    nao_status st = check_handle(g);
    if (st) return st;
    g->profiling = enable != 0;
    return NAO_OK;
}

nao_status nao_profile_read(nao_grid *g, nao_profile *out, int32_t reset) {
    nao_status st = check_handle(g);
    if (st) return st;
    DeviceGuard guard(g->device);
    NAO_CUDA(cudaDeviceSynchronize());
    for (auto &t : g->timed) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
            g->prof.ms[t.kid] += ms;
            g->prof.launches[t.kid] += 1;
        } else {
            cudaGetLastError();
        }
        g->event_pool.push_back(t.a);
        g->event_pool.push_back(t.b);
    }
    g->timed.clear();
    if (out) *out = g->prof;
    if (reset) g->prof = nao_profile{};
    return NAO_OK;
}

nao_status nao_sync_status(nao_grid *g) {
    nao_status st = check_handle(g);
    if (st) return st;
    DeviceGuard guard(g->device);
    // this handle's work only: its last call, then the error word on the setup stream
    if (g->used) NAO_CUDA(cudaEventSynchronize(g->ev_last));
    int32_t err[4] = {0, 0, 0, 0};
    NAO_CUDA(copy_async(err, g->d_err, sizeof(err), cudaMemcpyDeviceToHost, g->setup));
    NAO_CUDA(cudaStreamSynchronize(g->setup));
    if (err[0] != 0) {
        // reported once: the word is cleared so that the handle's later calls run again
        NAO_CUDA(cudaMemsetAsync(g->d_err, 0, sizeof(err), g->setup));
        NAO_CUDA(cudaStreamSynchronize(g->setup));
        return fail((nao_status)err[0], "device-side check failed (code " + std::to_string(err[1]) + ")");
    }
    return NAO_OK;
}

nao_status nao_fault_inject(const char *spec) {
    int kind;
    int64_t n;
    if (!parse_fault(spec, &kind, &n))
        return fail(NAO_ERR_INVALID_ARG, "fault spec must be alloc:<n>, copy:<n> or launch:<n> (n >= 1)");
    FaultState &F = faults();
    std::lock_guard<std::mutex> lock(F.mu);
    F.kind = kind;
    F.n = n;
    F.seen = 0;
    return NAO_OK;
}

nao_status nao_check_wait_timeout(nao_grid *g, int64_t max_cycles, void *cuda_stream) {
    nao_status st = check_handle(g);
    if (st) return st;
    if (max_cycles < 1 || max_cycles > (int64_t(1) << 34)) return fail(NAO_ERR_INVALID_ARG, "max_cycles outside 1..2^34");
    DeviceGuard guard(g->device);
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    CallEnd call_end(g, s);
    NAO_CUDA(launch_wait_timeout_probe(max_cycles, g->d_err, s));
    return mark_done(g, s);
}

const char *nao_status_string(nao_status s) {
    switch (s) {
        case NAO_OK: return "ok";
        case NAO_ERR_INVALID_ARG: return "invalid argument";
        case NAO_ERR_OUT_OF_MEMORY: return "out of memory";
        case NAO_ERR_CUDA: return "CUDA error";
        case NAO_ERR_TIMEOUT: return "device wait timed out";
        case NAO_ERR_INTERNAL: return "internal error";
        case NAO_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

const char *nao_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

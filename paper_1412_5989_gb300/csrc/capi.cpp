// The C ABI declared in include/cih.h: argument checks, error codes, and the
// order of device steps.  No C++ exception crosses it.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "cih_internal.h"

namespace cih {

static thread_local std::string g_detail;
static std::atomic<int64_t> g_launches{0};

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int fail(int code, const std::string &msg)
{
    g_detail = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    g_detail = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();
    return CIH_ERR_CUDA;
}

int device_pool(int device, cudaMemPool_t *pool)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    if (device < 0 || device >= 64) return fail(CIH_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaError_t e = cudaMemPoolCreate(&pools[device], &props);
        if (e != cudaSuccess) return cuda_fail(e, "memory pool");
        uint64_t keep = UINT64_MAX;                 // keep freed blocks for the next basis
        cudaMemPoolSetAttribute(pools[device], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    *pool = pools[device];
    return CIH_OK;
}

static double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static bool timing_on()
{
    static const bool on = std::getenv("CIH_TIMING") != nullptr;
    return on;
}

Timer::Timer(const char *w) : what(w), t0(now_ms()) {}
Timer::~Timer() { mark("end"); }
void Timer::mark_sync(const char *phase, cudaStream_t st)
{
    if (!timing_on()) return;
    cudaStreamSynchronize(st);
    mark(phase);
}

void Timer::mark(const char *phase)
{
    if (!timing_on()) return;
    double t = now_ms();
    std::fprintf(stderr, "[cih] %s: %s %.3f ms\n", what, phase, t - t0);
    t0 = t;
}

static void release(cih_basis *b)
{
    if (!b) return;
    int cur = 0;
    bool switched = false;
    if (!b->buffers.owned.empty() && cudaGetDevice(&cur) == cudaSuccess && cur != b->device)
        switched = cudaSetDevice(b->device) == cudaSuccess;
    if (!b->buffers.owned.empty()) {
        cudaDeviceSynchronize();                     // no kernel may still read the tables
        for (void *p : b->buffers.owned) cudaFreeAsync(p, 0);
        cudaStreamSynchronize(0);
    }
    if (switched) cudaSetDevice(cur);
    delete b;
}

template <class Fn>
static int guarded(Fn &&fn)
{
    try {
        return fn();
    } catch (const std::bad_alloc &) {
        return fail(CIH_ERR_NOMEM, "host allocation failed");
    } catch (...) {
        return fail(CIH_ERR_ARG, "unexpected host exception");
    }
}

}  // namespace cih

using namespace cih;

extern "C" {

int cih_basis_host_only(const cih_space_t *space, cih_basis_h *out)
{
    if (!space || !out) return fail(CIH_ERR_ARG, "NULL argument");
    *out = nullptr;
    return guarded([&]() -> int {
        cih_basis *b = new cih_basis;
        int rc = build_host_basis(*space, *b);
        if (rc) { release(b); return rc; }
        *out = b;
        return CIH_OK;
    });
}

int cih_basis_enumerate(const cih_space_t *space, cih_basis_h *out, void *stream)
{
    if (!space || !out) return fail(CIH_ERR_ARG, "NULL argument");
    *out = nullptr;
    return guarded([&]() -> int {
        cih_basis *b = new cih_basis;
        Timer tm("basis");
        int rc = build_host_species(*space, *b);
        tm.mark("host species");
        if (!rc) {
            cudaError_t e = cudaGetDevice(&b->device);
            rc = e == cudaSuccess ? upload_and_build_neighbours(*b, (cudaStream_t)stream,
                                                                [b]() { return build_host_rest(*b); })
                                  : cuda_fail(e, "cudaGetDevice");
        }
        if (rc) { release(b); return rc; }
        *out = b;
        return CIH_OK;
    });
}

int cih_basis_info(cih_basis_h h, int64_t *dim, int32_t *n_orb_p, int32_t *n_orb_n,
                   int64_t tbme_len[3], int64_t n_sd[2])
{
    if (!h) return fail(CIH_ERR_ARG, "NULL handle");
    if (dim) *dim = h->dim;
    if (n_orb_p) *n_orb_p = h->s[0].n_orb;
    if (n_orb_n) *n_orb_n = h->s[1].n_orb;
    if (tbme_len) for (int c = 0; c < 3; ++c) tbme_len[c] = h->layout.chan_len[c];
    if (n_sd) { n_sd[0] = h->s[0].n_sd; n_sd[1] = h->s[1].n_sd; }
    return CIH_OK;
}

int cih_basis_tables(cih_basis_h h, int32_t *orbitals, uint64_t *bits_p, uint64_t *bits_n,
                     int32_t *nbeg, int32_t *ncnt, int64_t *rowbase)
{
    if (!h) return fail(CIH_ERR_ARG, "NULL handle");
    if (orbitals) {
        int k = 0;
        for (int t = 0; t < 2; ++t)
            for (int a = 0; a < h->s[t].n_orb; ++a, ++k) {
                orbitals[4 * k] = h->s[t].oN[a];
                orbitals[4 * k + 1] = h->s[t].ol[a];
                orbitals[4 * k + 2] = h->s[t].oj2[a];
                orbitals[4 * k + 3] = h->s[t].om2[a];
            }
    }
    uint64_t *bits[2] = {bits_p, bits_n};
    for (int t = 0; t < 2; ++t)
        if (bits[t] && h->s[t].n_sd)
            std::memcpy(bits[t], h->s[t].bits.data(), sizeof(uint64_t) * kMaxWords * h->s[t].n_sd);
    if (nbeg && !h->nb.empty()) std::memcpy(nbeg, h->nb.data(), sizeof(int32_t) * h->nb.size());
    if (ncnt && !h->nc.empty()) std::memcpy(ncnt, h->nc.data(), sizeof(int32_t) * h->nc.size());
    if (rowbase) std::memcpy(rowbase, h->rowbase.data(), sizeof(int64_t) * h->rowbase.size());
    return CIH_OK;
}

int cih_tbme_index(cih_basis_h h, int32_t a, int32_t b, int32_t c, int32_t d, int64_t *index, int32_t *sign)
{
    if (!h || !index || !sign) return fail(CIH_ERR_ARG, "NULL argument");
    int ntot = h->s[0].n_orb + h->s[1].n_orb;
    *index = -1;
    *sign = 0;
    if (a < 0 || b < 0 || c < 0 || d < 0 || a >= ntot || b >= ntot || c >= ntot || d >= ntot) return CIH_OK;
    int32_t e1 = h->layout.pid[(size_t)a * ntot + b], e2 = h->layout.pid[(size_t)c * ntot + d];
    if (e1 < 0 || e2 < 0 || ((e1 >> 16) & 0xFFF) != ((e2 >> 16) & 0xFFF)) return CIH_OK;
    int g = (e1 >> 16) & 0xFFF;
    int64_t u = e1 & 0xFFFF, v = e2 & 0xFFFF;
    if (u > v) std::swap(u, v);
    int64_t n = h->layout.gsize[g];
    *index = h->layout.goff[g] + u * n - u * (u - 1) / 2 + (v - u);
    *sign = (((e1 ^ e2) >> 30) & 1) ? -1 : 1;
    return CIH_OK;
}

int cih_onebody_info(cih_basis_h h, int64_t *len)
{
    if (!h || !len) return fail(CIH_ERR_ARG, "NULL argument");
    *len = h->onebody.total;
    return CIH_OK;
}

int cih_onebody_index(cih_basis_h h, int32_t a, int32_t c, int64_t *index)
{
    if (!h || !index) return fail(CIH_ERR_ARG, "NULL argument");
    const int ntot = h->s[0].n_orb + h->s[1].n_orb;
    *index = -1;
    if (a < 0 || c < 0 || a >= ntot || c >= ntot) return CIH_OK;
    const OneBodyLayout &L = h->onebody;
    const int g = L.grp[a];
    if (g < 0 || g != L.grp[c]) return CIH_OK;
    int64_t u = L.loc[a], v = L.loc[c];
    if (u > v) std::swap(u, v);
    const int64_t n = L.gsize[g];
    *index = L.goff[g] + u * n - u * (u - 1) / 2 + (v - u);
    return CIH_OK;
}

int cih_basis_destroy(cih_basis_h h)
{
    if (!h) return fail(CIH_ERR_ARG, "NULL handle");
    release(h);
    return CIH_OK;
}

static int needs_device(cih_basis_h h)
{
    if (!h) return fail(CIH_ERR_ARG, "NULL handle");
    if (!h->dev_status) return fail(CIH_ERR_ARG, "host-only basis: build it with cih_basis_enumerate");
    return CIH_OK;
}

int cih_ham_count(cih_basis_h h, int64_t *rowptr_dev, int64_t *nnz_out, void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (!rowptr_dev) return fail(CIH_ERR_ARG, "NULL rowptr");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = launch_count(*h, rowptr_dev, st))) return rc;
    if ((rc = launch_scan(*h, rowptr_dev, st))) return rc;
    if (nnz_out) {
        cudaError_t e = cudaMemcpyAsync(nnz_out, rowptr_dev + h->dim, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "count: read nnz");
    }
    return CIH_OK;
}

int cih_ham_fill(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, double hbar_omega,
                 const float *tbme_dev, const double *e_sp_dev, int32_t *col_dev, float *val_dev, void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (!rowptr_dev || !col_dev || !val_dev || K < 1) return fail(CIH_ERR_ARG, "NULL array or K < 1");
    if (!tbme_dev && h->layout.total > 0) return fail(CIH_ERR_ARG, "NULL two-body table");
    return launch_fill(*h, rowptr_dev, K, hbar_omega, tbme_dev, false, false, e_sp_dev, col_dev, val_dev,
                       (cudaStream_t)stream);
}

int cih_ham_fill_onebody(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, const float *tbme_dev,
                         const double *onebody_dev, int32_t *col_dev, float *val_dev, void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (!rowptr_dev || !col_dev || !val_dev || !onebody_dev || K < 1) return fail(CIH_ERR_ARG, "NULL array or K < 1");
    if (!tbme_dev && h->layout.total > 0) return fail(CIH_ERR_ARG, "NULL two-body table");
    return launch_fill(*h, rowptr_dev, K, 0.0, tbme_dev, false, false, nullptr, col_dev, val_dev, (cudaStream_t)stream,
                       0, -1, false, onebody_dev);
}

int cih_ham_fill_rows(cih_basis_h h, const int64_t *rowptr_dev, int64_t r0, int64_t r1, int32_t K,
                      double hbar_omega, const float *tbme_dev, const double *e_sp_dev, int32_t *col_dev,
                      float *val_dev, void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (r0 < 0 || r1 < r0 || r1 > h->dim) return fail(CIH_ERR_ARG, "row range outside 0 .. dim");
    if (r1 == r0) return CIH_OK;
    if (!rowptr_dev || !col_dev || !val_dev || K < 1) return fail(CIH_ERR_ARG, "NULL array or K < 1");
    if (!tbme_dev && h->layout.total > 0) return fail(CIH_ERR_ARG, "NULL two-body table");
    return launch_fill(*h, rowptr_dev, K, hbar_omega, tbme_dev, false, false, e_sp_dev, col_dev, val_dev,
                       (cudaStream_t)stream, r0, r1, true);
}

int cih_shard_rows(const int64_t *rowptr_host, int64_t dim, int32_t nshards, int64_t *bounds_host)
{
    if (!rowptr_host || !bounds_host || dim < 0 || nshards < 1) return fail(CIH_ERR_ARG, "bad shard arguments");
    const int64_t nnz = rowptr_host[dim];
    bounds_host[0] = 0;
    for (int32_t k = 1; k < nshards; ++k) {
        // first row whose elements start at or after the k-th equal share of the nonzeros
        const int64_t target = (int64_t)((__int128)nnz * k / nshards);
        const int64_t r = std::lower_bound(rowptr_host, rowptr_host + dim, target) - rowptr_host;
        bounds_host[k] = std::max(bounds_host[k - 1], std::min(r, dim));
    }
    bounds_host[nshards] = dim;
    return CIH_OK;
}

int cih_ham_fill_interleaved(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, double hbar_omega,
                             const float *tbme_il_dev, const double *e_sp_dev, int32_t *col_dev, float *val_dev,
                             void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (!rowptr_dev || !col_dev || !val_dev || K < 1) return fail(CIH_ERR_ARG, "NULL array or K < 1");
    if (!tbme_il_dev && h->layout.total > 0) return fail(CIH_ERR_ARG, "NULL two-body table");
    return launch_fill(*h, rowptr_dev, K, hbar_omega, tbme_il_dev, true, false, e_sp_dev, col_dev, val_dev,
                       (cudaStream_t)stream);
}

int cih_ham_fill_batched(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, double hbar_omega,
                         const float *tbme_il_dev, const double *e_sp_dev, int32_t *col_dev, float *val_em_dev,
                         void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (!rowptr_dev || !col_dev || !val_em_dev || K < 1) return fail(CIH_ERR_ARG, "NULL array or K < 1");
    if (!tbme_il_dev && h->layout.total > 0) return fail(CIH_ERR_ARG, "NULL two-body table");
    return launch_fill(*h, rowptr_dev, K, hbar_omega, tbme_il_dev, true, true, e_sp_dev, col_dev, val_em_dev,
                       (cudaStream_t)stream);
}

int cih_ham_build_host(cih_basis_h h, int32_t K, double hbar_omega, const float *tbme_host, const double *e_sp_host,
                       int64_t *rowptr_host, int32_t *col_host, float *val_host, int64_t capacity, int64_t *nnz_out,
                       void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (K < 1 || K > 256 || !rowptr_host || !col_host || !val_host || capacity < 0 ||
        (!tbme_host && h->layout.total > 0))
        return fail(CIH_ERR_ARG, "build_host: K, host arrays or capacity");
    return guarded([&]() -> int {
        return build_host(*h, K, hbar_omega, tbme_host, e_sp_host, rowptr_host, col_host, val_host, capacity, nnz_out,
                          (cudaStream_t)stream);
    });
}

int cih_tbme_interleave(int32_t K, int64_t tbme_len, const float *tbme_dev, float *tbme_il_dev, void *stream)
{
    if (K < 1 || tbme_len < 0 || (tbme_len > 0 && (!tbme_dev || !tbme_il_dev)))
        return fail(CIH_ERR_ARG, "bad interleave arguments");
    return launch_interleave(K, tbme_len, tbme_dev, tbme_il_dev, (cudaStream_t)stream);
}

int cih_set_launch(cih_basis_h h, int32_t warps_per_cta, int32_t ctas_per_sm)
{
    if (!h) return fail(CIH_ERR_ARG, "NULL handle");
    if ((warps_per_cta != 8 && warps_per_cta != 16) || ctas_per_sm < 0 || ctas_per_sm > 32)
        return fail(CIH_ERR_ARG, "warps_per_cta must be 8 or 16, ctas_per_sm 0..32");
    h->launch_warps = warps_per_cta;
    h->launch_ctas = ctas_per_sm;
    return CIH_OK;
}

int cih_set_count_mode(cih_basis_h h, int32_t walk)
{
    if (!h) return fail(CIH_ERR_ARG, "NULL handle");
    if (walk != 0 && walk != 1) return fail(CIH_ERR_ARG, "count mode must be 0 (count lists) or 1 (walk)");
    h->count_walk = walk;
    return CIH_OK;
}

int cih_autotune_fill(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, double hbar_omega, const float *tbme_dev,
                      int32_t interleaved, const double *e_sp_dev, int32_t *col_dev, float *val_dev, void *stream,
                      int32_t *best_warps, int32_t *best_ctas, float *best_ms)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (!rowptr_dev || !col_dev || !val_dev || K < 1) return fail(CIH_ERR_ARG, "NULL array or K < 1");
    cudaStream_t st = (cudaStream_t)stream;
    const int warps[2] = {16, 8};
    const int ctas[4] = {0, 1, 2, 3};
    float best = 1e30f;
    int bw = 16, bc = 0;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "autotune events");
    for (int wi = 0; wi < 2 && !rc; ++wi)
        for (int ci = 0; ci < 4 && !rc; ++ci) {
            h->launch_warps = warps[wi];
            h->launch_ctas = ctas[ci];
            float ms = 0.0f, tmin = 1e30f;
            for (int rep = 0; rep < 3 && !rc; ++rep) {
                cudaEventRecord(e0, st);
                rc = launch_fill(*h, rowptr_dev, K, hbar_omega, tbme_dev, interleaved != 0, interleaved == 2, e_sp_dev,
                                 col_dev, val_dev, st);
                cudaEventRecord(e1, st);
                if (!rc && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
                    rep > 0)
                    tmin = std::min(tmin, ms);
            }
            if (!rc && tmin < best) { best = tmin; bw = warps[wi]; bc = ctas[ci]; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->launch_warps = bw;
    h->launch_ctas = bc;
    if (best_warps) *best_warps = bw;
    if (best_ctas) *best_ctas = bc;
    if (best_ms) *best_ms = best;
    return rc;
}

int cih_check(cih_basis_h h, void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    int st4[4] = {0, 0, 0, 0};
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(st4, h->dev_status, sizeof(st4), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dev_status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dev_status + 2, 0, 2 * sizeof(int), st);
    const int status = st4[0];
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "check");
    if (status)
        return fail(CIH_ERR_DEVICE, std::string("device status bits ") + std::to_string(status) +
                                        " (1: pair outside the table layout, 2: write beyond the row, "
                                        "4: two-move index, 8: deferred queue, 32: adjoint vector not normalised (an entry of magnitude 4 "
                                        "or more, or a squared norm above 1 + 1e-6)); first: " + std::to_string(st4[2]) + " " +
                                        std::to_string(st4[3]));
    return CIH_OK;
}

static int lanczos_entry(cih_basis_h h, const int64_t *rowptr_dev, const int32_t *col_dev, const float *val_dev,
                         int32_t K, int32_t nev, int32_t max_iter, double tol, double *evals_host,
                         double *evec0_dev, void *stream, bool values_em)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (!rowptr_dev || !col_dev || !val_dev || !evals_host) return fail(CIH_ERR_ARG, "NULL array");
    if (K < 1 || K > 256 || nev < 1 || nev > 64 || max_iter < 1 || max_iter > 2048 || !(tol > 0))
        return fail(CIH_ERR_ARG, "K, nev, max_iter or tol out of range");
    return guarded([&]() -> int {
        return lanczos(*h, rowptr_dev, col_dev, val_dev, K, nev, max_iter, tol, evals_host, evec0_dev,
                       (cudaStream_t)stream, values_em);
    });
}

int cih_lanczos_lowest(cih_basis_h h, const int64_t *rowptr_dev, const int32_t *col_dev,
                       const float *val_dev, int32_t K, int32_t nev, int32_t max_iter, double tol,
                       double *evals_host, double *evec0_dev, void *stream)
{
    return lanczos_entry(h, rowptr_dev, col_dev, val_dev, K, nev, max_iter, tol, evals_host, evec0_dev, stream, false);
}

int cih_lanczos_lowest_em(cih_basis_h h, const int64_t *rowptr_dev, const int32_t *col_dev,
                          const float *val_em_dev, int32_t K, int32_t nev, int32_t max_iter, double tol,
                          double *evals_host, double *evec0_dev, void *stream)
{
    return lanczos_entry(h, rowptr_dev, col_dev, val_em_dev, K, nev, max_iter, tol, evals_host, evec0_dev, stream,
                         true);
}

int cih_ham_spmv(cih_basis_h h, const int64_t *rowptr_dev, const int32_t *col_dev, const float *val_dev,
                 int32_t K, int32_t values_em, const double *x_dev, double *y_dev, void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (K < 1 || K > 256 || (values_em != 0 && values_em != 1)) return fail(CIH_ERR_ARG, "K or values_em out of range");
    if (h->dim == 0) return CIH_OK;                               // nothing to multiply
    if (!rowptr_dev || !col_dev || !val_dev || !x_dev || !y_dev) return fail(CIH_ERR_ARG, "NULL array");
    if (x_dev == y_dev) return fail(CIH_ERR_ARG, "x and y must not be the same array");
    return guarded([&]() -> int {
        return ham_spmv(*h, rowptr_dev, col_dev, val_dev, K, values_em != 0, x_dev, y_dev, (cudaStream_t)stream);
    });
}

int cih_ham_upper_sumsq(cih_basis_h h, const int64_t *rowptr_dev, int64_t r0, int64_t r1, const float *val_dev,
                        int32_t K, int32_t values_em, double *f2_host, void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (!f2_host) return fail(CIH_ERR_ARG, "NULL output");
    *f2_host = 0.0;
    if (K < 1 || K > 256 || (values_em != 0 && values_em != 1)) return fail(CIH_ERR_ARG, "K or values_em out of range");
    if (r0 < 0 || r1 < r0 || r1 > h->dim) return fail(CIH_ERR_ARG, "row range outside 0 .. dim");
    if (r1 == r0) return CIH_OK;
    if (!rowptr_dev || !val_dev) return fail(CIH_ERR_ARG, "NULL array");
    return guarded([&]() -> int {
        return upper_sumsq(*h, rowptr_dev, r0, r1, val_dev, K, values_em != 0, f2_host, (cudaStream_t)stream);
    });
}

int cih_lanczos_lowest_shard(cih_basis_h h, const int64_t *rowptr_dev, int64_t r0, int64_t r1, const int32_t *col_dev,
                             const float *val_dev, int32_t K, int32_t values_em, int32_t nev, int32_t max_iter,
                             double tol, double f2, uint64_t *acc_dev, double *yx_dev, int (*combine)(void *),
                             void *ctx, double *evals_host, double *evec0_dev, void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (!rowptr_dev || !evals_host || !acc_dev || !yx_dev || !combine) return fail(CIH_ERR_ARG, "NULL array or callback");
    if (K < 1 || K > 256 || nev < 1 || nev > 64 || max_iter < 1 || max_iter > 2048 || !(tol > 0) ||
        (values_em != 0 && values_em != 1) || !(f2 >= 0))
        return fail(CIH_ERR_ARG, "K, nev, max_iter, tol, values_em or f2 out of range");
    if (r0 < 0 || r1 < r0 || r1 > h->dim) return fail(CIH_ERR_ARG, "row range outside 0 .. dim");
    if (r1 > r0 && (!col_dev || !val_dev)) return fail(CIH_ERR_ARG, "NULL array");
    ShardRun sh;
    sh.r0 = r0;
    sh.r1 = r1;
    sh.f2 = f2;
    sh.acc = reinterpret_cast<unsigned long long *>(acc_dev);
    sh.yx = yx_dev;
    sh.combine = combine;
    sh.ctx = ctx;
    return guarded([&]() -> int {
        return lanczos(*h, rowptr_dev, col_dev, val_dev, K, nev, max_iter, tol, evals_host, evec0_dev,
                       (cudaStream_t)stream, values_em != 0, &sh);
    });
}

int cih_ham_tbme_grad(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, const double *psi_dev,
                      double *grad_dev, void *stream)
{
    int rc = needs_device(h);
    if (rc) return rc;
    if (!psi_dev || !grad_dev || K < 1) return fail(CIH_ERR_ARG, "NULL array or K < 1");
    int64_t n = (int64_t)K * h->layout.total;
    if (n == 0) return CIH_OK;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long *acc = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&acc, sizeof(unsigned long long) * n, h->pool, st);
    if (e != cudaSuccess) return fail(CIH_ERR_NOMEM, std::string("gradient scratch: ") + cudaGetErrorString(e));
    e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * n, st);
    if (e != cudaSuccess) rc = cuda_fail(e, "gradient scratch clear");
    if (!rc) rc = launch_grad(*h, rowptr_dev, K, psi_dev, acc, st);
    if (!rc) rc = launch_grad_finish(n, acc, grad_dev, st);
    cudaFreeAsync(acc, st);
    return rc;
}

int cih_batch_solve(cih_instance_t *inst, int32_t n, double hbar_omega, int32_t nev, int32_t max_iter, double tol,
                    int64_t hbm_budget, void *stream)
{
    if (n < 0 || (n > 0 && !inst)) return fail(CIH_ERR_ARG, "NULL instance array");
    if (n > 256) return fail(CIH_ERR_UNSUPPORTED, "at most 256 instances per batch");
    if (nev < 1 || nev > 64 || max_iter < 1 || max_iter > 2048 || !(tol > 0) || hbm_budget < 0)
        return fail(CIH_ERR_ARG, "nev, max_iter, tol or budget out of range");
    for (int i = 0; i < n; ++i) {
        const cih_instance_t &x = inst[i];
        int rc = needs_device(x.basis);
        if (rc) return rc;
        if (x.K < 1 || x.K > 256 || !x.evals_host || (!x.tbme_dev && x.basis->layout.total > 0))
            return fail(CIH_ERR_ARG, "instance " + std::to_string(i) + ": K, tables or eigenvalue array");
        if (x.basis->device != inst[0].basis->device)
            return fail(CIH_ERR_ARG, "instances on different devices");
    }
    if (n == 0) return CIH_OK;
    return guarded([&]() -> int {
        return batch_solve(inst, n, hbar_omega, nev, max_iter, tol, hbm_budget, (cudaStream_t)stream);
    });
}

const char *cih_strerror(int code)
{
    switch (code) {
    case CIH_OK: return "ok";
    case CIH_ERR_ARG: return "invalid argument";
    case CIH_ERR_NOMEM: return "out of memory";
    case CIH_ERR_CAPACITY: return "result does not fit the capacity";
    case CIH_ERR_TIMEOUT: return "bounded device wait timed out";
    case CIH_ERR_UNSUPPORTED: return "size outside what the kernels handle";
    case CIH_ERR_CUDA: return "CUDA runtime error";
    case CIH_ERR_DEVICE: return "device-side check failed";
    default: return "unknown error";
    }
}

const char *cih_last_error_detail(void) { return g_detail.c_str(); }

int cih_kernel_launches(int64_t *out)
{
    if (!out) return fail(CIH_ERR_ARG, "NULL argument");
    *out = g_launches.load(std::memory_order_relaxed);
    return CIH_OK;
}

}  // extern "C"

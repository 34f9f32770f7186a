// cih_ham_build_host: the two-body tables from host memory in, the half-stored
// matrix (Sec. 2, stored in compressed rows as in Sec. 4.1) out to host
// memory, with the copies inside the call and the device-to-host copy of each
// row chunk overlapped with the fill of the next one.
#include <algorithm>
#include <vector>

#include "cih_internal.h"

namespace cih {

int build_host(cih_basis &b, int K, double hw, const float *tbme_h, const double *esp_h, int64_t *rowptr_h,
               int32_t *col_h, float *val_h, int64_t capacity, int64_t *nnz_out, cudaStream_t st)
{
    const int64_t dim = b.dim, tl = b.layout.total;
    const int n_orb = b.s[0].n_orb + b.s[1].n_orb;
    Timer tm("build_host");
    std::vector<void *> bufs;
    auto alloc = [&](void **p, size_t bytes) -> bool {
        // the library pool keeps the blocks mapped for the next call
        if (cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), b.pool, st) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        bufs.push_back(*p);
        return true;
    };
    cudaStream_t cs = nullptr;
    std::vector<cudaEvent_t> evs;
    int rc = CIH_OK;
    float *tbme_d = nullptr;
    double *esp_d = nullptr;
    int64_t *rowptr_d = nullptr;
    int32_t *col_d = nullptr;
    float *val_d = nullptr;
    int64_t nnz = 0;
    cudaError_t e;
    if (!alloc((void **)&tbme_d, sizeof(float) * (size_t)K * tl) || !alloc((void **)&rowptr_d, sizeof(int64_t) * (dim + 1)) ||
        (esp_h && !alloc((void **)&esp_d, sizeof(double) * n_orb))) {
        rc = fail(CIH_ERR_NOMEM, "build_host: device tables");
        goto done;
    }
    if (tl > 0) cudaMemcpyAsync(tbme_d, tbme_h, sizeof(float) * (size_t)K * tl, cudaMemcpyHostToDevice, st);
    if (esp_h) cudaMemcpyAsync(esp_d, esp_h, sizeof(double) * n_orb, cudaMemcpyHostToDevice, st);
    if ((rc = launch_count(b, rowptr_d, st)) || (rc = launch_scan(b, rowptr_d, st))) goto done;
    e = cudaMemcpyAsync(rowptr_h, rowptr_d, sizeof(int64_t) * (dim + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { rc = cuda_fail(e, "build_host: row pointers"); goto done; }
    nnz = rowptr_h[dim];
    if (nnz_out) *nnz_out = nnz;
    tm.mark("tables in, count, row pointers out");
    if (nnz > capacity) {
        rc = fail(CIH_ERR_CAPACITY, "build_host: " + std::to_string(nnz) + " stored nonzeros, capacity " +
                                        std::to_string(capacity));
        goto done;
    }
    if (!alloc((void **)&col_d, sizeof(int32_t) * (size_t)nnz) || !alloc((void **)&val_d, sizeof(float) * (size_t)K * nnz)) {
        rc = fail(CIH_ERR_NOMEM, "build_host: device matrix");
        goto done;
    }
    tm.mark_sync("device matrix allocated", st);
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) { cs = nullptr; rc = cuda_fail(e, "build_host: copy stream"); goto done; }
    {
        // row chunks of about equal nonzero counts; chunk c's copies wait for its fill
        const int C = (int)std::max<int64_t>(1, std::min<int64_t>(8, dim));
        std::vector<int64_t> rb(C + 1, dim);
        rb[0] = 0;
        for (int c = 1; c < C; ++c)
            rb[c] = std::lower_bound(rowptr_h, rowptr_h + dim + 1, nnz * c / C) - rowptr_h;
        for (int c = 0; c < C && !rc; ++c) {
            const int64_t r0 = std::min(rb[c], dim), r1 = std::max(r0, std::min(rb[c + 1], dim));
            if ((rc = launch_fill(b, rowptr_d, K, hw, tbme_d, false, false, esp_d, col_d, val_d, st, r0, r1))) break;
            cudaEvent_t ev;
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
                rc = cuda_fail(e, "build_host: event");
                break;
            }
            evs.push_back(ev);
            cudaEventRecord(ev, st);
            cudaStreamWaitEvent(cs, ev, 0);
            const int64_t e0 = rowptr_h[r0], e1 = rowptr_h[r1];
            if (e1 > e0) {
                cudaMemcpyAsync(col_h + e0, col_d + e0, sizeof(int32_t) * (e1 - e0), cudaMemcpyDeviceToHost, cs);
                for (int k = 0; k < K; ++k)
                    cudaMemcpyAsync(val_h + (int64_t)k * capacity + e0, val_d + (int64_t)k * nnz + e0,
                                    sizeof(float) * (e1 - e0), cudaMemcpyDeviceToHost, cs);
            }
        }
        tm.mark_sync("fill chunks done", st);
        e = cudaStreamSynchronize(cs);
        tm.mark("copies done");
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "build_host: copies");
        e = cudaGetLastError();
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "build_host");
    }
done:
    for (void *p : bufs) cudaFreeAsync(p, st);
    e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "build_host");
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
    return rc;
}

}  // namespace cih

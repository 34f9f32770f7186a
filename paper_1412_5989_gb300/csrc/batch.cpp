// cih_batch_solve: count, admit by device memory, build, Lanczos and adjoint
// for a batch of instances of different sizes (Sec. 4.1: nonzeros counted
// first so the arrays can be sized; Sec. 2: Lanczos on each matrix).
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "cih_internal.h"

namespace cih {
namespace {

struct Plan {
    int64_t resident = 0;   // col, values, Ritz vectors: held while the wave runs
    int64_t scratch = 0;    // Lanczos or adjoint scratch: one instance at a time
};

// device memory of one wave, released in one place
struct WaveMem {
    cudaStream_t st;
    cudaMemPool_t pool;
    std::vector<void *> ptrs;
    WaveMem(cudaStream_t s, cudaMemPool_t p) : st(s), pool(p) {}
    bool get(void **p, size_t bytes)
    {
        if (cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, st) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        ptrs.push_back(*p);
        return true;
    }
    ~WaveMem()
    {
        for (void *p : ptrs) cudaFreeAsync(p, st);
    }
};

// streams and events of the concurrent branches, created before any capture
struct Branches {
    std::vector<cudaStream_t> s;
    std::vector<cudaEvent_t> done;
    cudaEvent_t fork = nullptr;
    int make(int n)
    {
        if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess) return -1;
        for (int i = 0; i < n; ++i) {
            cudaStream_t x;
            cudaEvent_t e;
            if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) return -1;
            s.push_back(x);
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return -1;
            done.push_back(e);
        }
        return 0;
    }
    ~Branches()
    {
        for (cudaEvent_t e : done) cudaEventDestroy(e);
        for (cudaStream_t x : s) cudaStreamDestroy(x);
        if (fork) cudaEventDestroy(fork);
    }
};

// run fn(i, stream_i) for each i in idx on its own branch forked from `st`
// and joined back into it; with as_graph the branches are recorded into a
// CUDA graph that is launched once on `st`
template <class Fn>
int fan_out(cudaStream_t st, const std::vector<int> &idx, Branches &br, bool as_graph, Fn &&fn)
{
    cudaStream_t origin = st;
    cudaStream_t cap = nullptr;
    if (as_graph) {
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail(cudaGetLastError(), "batch: capture stream");
        cudaEvent_t ready;
        cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
        cudaEventRecord(ready, st);                   // the capture stream starts after st's prior work
        cudaStreamWaitEvent(cap, ready, 0);
        cudaEventDestroy(ready);
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            return cuda_fail(e, "batch: begin capture");
        }
        origin = cap;
    }
    int rc = CIH_OK;
    cudaEventRecord(br.fork, origin);
    for (size_t q = 0; q < idx.size() && !rc; ++q) {
        cudaStreamWaitEvent(br.s[q], br.fork, 0);
        rc = fn(idx[q], br.s[q]);
        cudaEventRecord(br.done[q], br.s[q]);
        cudaStreamWaitEvent(origin, br.done[q], 0);
    }
    if (as_graph) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(cap, &g);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "batch: end capture");
        cudaGraphExec_t x = nullptr;
        if (!rc) {
            e = cudaGraphInstantiate(&x, g, 0);
            if (e != cudaSuccess) rc = cuda_fail(e, "batch: graph instantiate");
        }
        if (!rc) {                                    // (the fills were counted as they were captured)
            e = cudaGraphLaunch(x, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "batch: graph launch");
        }
        if (x) cudaGraphExecDestroy(x);               // deferred by the runtime until the launch completes
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cap);
    }
    return rc;
}

}  // namespace

int batch_solve(cih_instance_t *inst, int n, double hw, int nev, int max_iter, double tol, int64_t budget,
                cudaStream_t st)
{
    for (int i = 0; i < n; ++i) {
        inst[i].nnz = 0;
        inst[i].bytes = 0;
        inst[i].wave = -1;
        inst[i].status = CIH_OK;
    }
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        cudaError_t e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) return cuda_fail(e, "batch: memory info");
        budget = (int64_t)(0.9 * (double)fr);
    }
    Branches br;
    if (br.make(n)) return cuda_fail(cudaGetLastError(), "batch: streams");
    for (int i = 0; i < n; ++i) {
        const int rc = prepare_rows(*inst[i].basis, inst[i].K);
        if (rc) return rc;
    }

    // 1. counts and row pointers of every instance
    const cudaMemPool_t pool = inst[0].basis->pool;
    WaveMem keep(st, pool);
    std::vector<int64_t *> rowptr(n, nullptr);
    int64_t rowptr_bytes = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t b = 8 * (inst[i].basis->dim + 1);
        if (!keep.get((void **)&rowptr[i], b)) return fail(CIH_ERR_NOMEM, "batch: row pointers");
        rowptr_bytes += b;
    }
    std::vector<int> all(n);
    for (int i = 0; i < n; ++i) all[i] = i;
    // a basis given twice would share its scan scratch: then the counts run one after another
    bool distinct = true;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j) distinct = distinct && inst[i].basis != inst[j].basis;
    auto count = [&](int i, cudaStream_t s) {
        int r = launch_count(*inst[i].basis, rowptr[i], s);
        return r ? r : launch_scan(*inst[i].basis, rowptr[i], s);
    };
    int rc = CIH_OK;
    if (distinct) rc = fan_out(st, all, br, false, count);
    for (int i = 0; i < n && !distinct && !rc; ++i) rc = count(i, st);
    if (rc) return rc;
    std::vector<int64_t> nnz(n, 0);
    for (int i = 0; i < n; ++i) {
        cudaError_t e = cudaMemcpyAsync(&nnz[i], rowptr[i] + inst[i].basis->dim, sizeof(int64_t),
                                        cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch: read counts");
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "batch: counts");

    // 2. bytes per instance
    std::vector<Plan> plan(n);
    for (int i = 0; i < n; ++i) {
        const cih_basis &b = *inst[i].basis;
        const int64_t K = inst[i].K;
        inst[i].nnz = nnz[i];
        plan[i].resident = 4 * std::max<int64_t>(nnz[i], 1) + 4 * K * std::max<int64_t>(nnz[i], 1) + 8 * K * b.dim + 3 * 256;
        const int64_t grad = inst[i].grad_dev ? 8 * K * b.layout.total : 0;
        plan[i].scratch = std::max(lanczos_bytes(b.dim, nnz[i], (int)K, max_iter), grad);
        inst[i].bytes = 8 * (b.dim + 1) + plan[i].resident + plan[i].scratch;
    }

    // 3. waves in the given order: resident sum + the largest scratch within the budget
    const int64_t avail = budget - rowptr_bytes;
    std::vector<std::vector<int>> waves;
    int64_t res = 0, scr = 0;
    for (int i = 0; i < n; ++i) {
        if (plan[i].resident + plan[i].scratch > avail) {
            inst[i].status = CIH_ERR_CAPACITY;
            continue;
        }
        if (waves.empty() || res + plan[i].resident + std::max(scr, plan[i].scratch) > avail) {
            waves.emplace_back();
            res = scr = 0;
        }
        waves.back().push_back(i);
        res += plan[i].resident;
        scr = std::max(scr, plan[i].scratch);
        inst[i].wave = (int)waves.size() - 1;
    }

    // 4. per wave: one graph of fills, then Lanczos and the adjoint per instance
    for (const std::vector<int> &w : waves) {
        WaveMem mem(st, pool);
        std::vector<int32_t *> col(n, nullptr);
        std::vector<float *> val(n, nullptr);
        std::vector<double *> psi(n, nullptr);
        for (int i : w) {
            const int64_t K = inst[i].K, m = std::max<int64_t>(nnz[i], 1);
            if (!mem.get((void **)&col[i], 4 * m) || !mem.get((void **)&val[i], 4 * K * m) ||
                !mem.get((void **)&psi[i], 8 * K * std::max<int64_t>(inst[i].basis->dim, 1)))
                return fail(CIH_ERR_NOMEM, "batch: wave arrays");
        }
        rc = fan_out(st, w, br, true, [&](int i, cudaStream_t s) {
            return launch_fill(*inst[i].basis, rowptr[i], inst[i].K, hw, inst[i].tbme_dev, false, false, inst[i].e_sp_dev,
                               col[i], val[i], s);
        });
        if (rc) return rc;
        for (int i : w) {
            const cih_basis &b = *inst[i].basis;
            const int r = lanczos(b, rowptr[i], col[i], val[i], inst[i].K, nev, max_iter, tol, inst[i].evals_host,
                                  psi[i], st);
            if (r < 0) return r;
            inst[i].status = r;
            if (inst[i].grad_dev && b.layout.total > 0) {
                const int64_t ng = (int64_t)inst[i].K * b.layout.total;
                unsigned long long *acc = nullptr;
                e = cudaMallocFromPoolAsync((void **)&acc, sizeof(unsigned long long) * ng, pool, st);
                if (e != cudaSuccess) return fail(CIH_ERR_NOMEM, "batch: adjoint scratch");
                e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * ng, st);
                int g = e == cudaSuccess ? CIH_OK : cuda_fail(e, "batch: adjoint clear");
                if (!g) g = launch_grad(b, rowptr[i], inst[i].K, psi[i], acc, st);
                if (!g) g = launch_grad_finish(ng, acc, inst[i].grad_dev, st);
                cudaFreeAsync(acc, st);
                if (g) return g;
            }
        }
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "batch: wave");
    }
    for (int i = 0; i < n; ++i)
        if (inst[i].status != CIH_OK) return 1;
    return CIH_OK;
}

}  // namespace cih

// Lanczos for the lowest eigenpairs (Sec. 2: successive matrix-vector
// products and orthogonalisations).  Device: half-symmetric SpMV with FP32
// values and FP64 accumulation, FP64 Lanczos vectors, full
// reorthogonalisation (classical Gram-Schmidt, applied twice) with
// deterministic two-stage reductions.  Host: the symmetric tridiagonal
// eigenproblem by implicit-shift QR with Wilkinson shifts.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "cih_internal.h"


namespace cih {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 304;            // partial sums per reduction

// y = H x for the stored upper triangle: row part accumulated in FP64 per
// warp, the mirrored part added to y[j] atomically.
__global__ void k_spmv_half(int64_t dim, const int64_t *rowptr, const int32_t *col, const float *val,
                            const double *x, double *y)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < dim; i += nw) {
        int64_t b = rowptr[i], e = rowptr[i + 1];
        double xi = x[i], acc = 0.0;
        for (int64_t k = b + lane; k < e; k += 32) {
            int64_t j = col[k];
            double h = val[k];
            acc += h * x[j];
            if (j != i) atomicAdd(y + j, h * xi);
        }
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
        if (lane == 0) atomicAdd(y + i, acc);
    }
}

// partial[r * kRedBlocks + blk] = sum_i V[r][i] * w[i] over this block's slice
__global__ void k_multidot(int64_t dim, int nvec, const double *V, const double *w, double *partial)
{
    __shared__ double red[kRedThreads / 32];
    for (int r = blockIdx.y; r < nvec; r += gridDim.y) {
        const double *v = V + (int64_t)r * dim;
        double acc = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < dim; i += (int64_t)gridDim.x * kRedThreads)
            acc += v[i] * w[i];
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            double s = threadIdx.x < kRedThreads / 32 ? red[threadIdx.x] : 0.0;
            for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
            if (threadIdx.x == 0) partial[(int64_t)r * gridDim.x + blockIdx.x] = s;
        }
        __syncthreads();
    }
}

// out[r] = sum of partial[r][*] in a fixed order
__global__ void k_finish_dots(int nvec, int nparts, const double *partial, double *out)
{
    int r = blockIdx.x;
    if (r >= nvec) return;
    __shared__ double red[32];
    double s = 0.0;
    for (int k = threadIdx.x; k < nparts; k += 32) s += partial[(int64_t)r * nparts + k];
    red[threadIdx.x] = s;
    __syncwarp();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < 32; ++k) t += red[k];
        out[r] = t;
    }
}

// w -= sum_r coef[r] V[r]
__global__ void k_subtract(int64_t dim, int nvec, const double *V, const double *coef, double *w)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
        double s = w[i];
        for (int r = 0; r < nvec; ++r) s -= coef[r] * V[(int64_t)r * dim + i];
        w[i] = s;
    }
}

// out[i] = sum_r coef[r] V[r][i] (Ritz vector)
__global__ void k_combine(int64_t dim, int nvec, const double *V, const double *coef, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < nvec; ++r) s += coef[r] * V[(int64_t)r * dim + i];
        out[i] = s;
    }
}

__global__ void k_scale(int64_t dim, const double *in, double f, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] * f;
}

// deterministic start vector: 1 + 0.5 u_i with u_i from the splitmix64 hash of i
__global__ void k_start(int64_t dim, double *v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)i + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        v[i] = 1.0 + 0.5 * (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
}

int grid1(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
}

}  // namespace

int lanczos(const cih_basis &b, const int64_t *rowptr, const int32_t *col, const float *val, int K, int nev,
            int max_iter, double tol, double *evals, double *evec0, cudaStream_t st)
{
    const int64_t dim = b.dim;
    for (int k = 0; k < K * nev; ++k) evals[k] = NAN;
    if (dim == 0) return CIH_OK;
    int64_t nnz = 0;
    cudaError_t e = cudaMemcpyAsync(&nnz, rowptr + dim, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "lanczos: read nnz");
    const int m_max = (int)std::min<int64_t>(max_iter, dim);
    double *V = nullptr, *w = nullptr, *partial = nullptr, *coef = nullptr;
    size_t vbytes = sizeof(double) * (size_t)(m_max + 1) * dim;
    e = cudaMallocAsync((void **)&V, vbytes, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&w, sizeof(double) * dim, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&partial, sizeof(double) * (size_t)(m_max + 1) * kRedBlocks, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&coef, sizeof(double) * (m_max + 1), st);
    if (e != cudaSuccess) {
        cudaFreeAsync(V, st); cudaFreeAsync(w, st); cudaFreeAsync(partial, st); cudaFreeAsync(coef, st);
        return fail(CIH_ERR_NOMEM, "lanczos vectors");
    }
    int rc = CIH_OK, not_converged = 0;
    const int g = grid1(dim);
    auto dots = [&](int nvec, double *out_dev) {
        dim3 grid(kRedBlocks, std::min(nvec, 65535));
        count_launches(1);
        k_multidot<<<grid, kRedThreads, 0, st>>>(dim, nvec, V, w, partial);
        count_launches(1);
        k_finish_dots<<<nvec, 32, 0, st>>>(nvec, kRedBlocks, partial, out_dev);
    };
    std::vector<double> alpha, beta, hcoef(m_max + 1), Z;
    for (int set = 0; set < K && rc == CIH_OK; ++set) {
        const float *vk = val + (int64_t)set * nnz;
        alpha.clear();
        beta.clear();
        // v0 = start / |start|
        count_launches(1);
        k_start<<<g, 256, 0, st>>>(dim, w);
        {
            // norm of the start vector via a one-vector dot of w with itself
            count_launches(1);
            k_scale<<<g, 256, 0, st>>>(dim, w, 1.0, V);
            dim3 grid(kRedBlocks, 1);
            count_launches(1);
            k_multidot<<<grid, kRedThreads, 0, st>>>(dim, 1, V, w, partial);
            count_launches(1);
            k_finish_dots<<<1, 32, 0, st>>>(1, kRedBlocks, partial, coef);
            double nrm2 = 0.0;
            cudaMemcpyAsync(&nrm2, coef, sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            count_launches(1);
            k_scale<<<g, 256, 0, st>>>(dim, w, 1.0 / std::sqrt(nrm2), V);
        }
        int m = 0;
        bool conv = false;
        std::vector<double> theta;
        for (int j = 0; j < m_max; ++j) {
            double *vj = V + (int64_t)j * dim;
            cudaMemsetAsync(w, 0, sizeof(double) * dim, st);
            count_launches(1);
            k_spmv_half<<<(int)std::min<int64_t>((dim + 7) / 8, 152 * 32), 256, 0, st>>>(dim, rowptr, col, vk, vj, w);
            // alpha_j = v_j . w, then two classical Gram-Schmidt passes
            for (int pass = 0; pass < 2; ++pass) {
                dots(j + 1, coef);
                if (pass == 0) {
                    cudaMemcpyAsync(hcoef.data(), coef, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, st);
                    cudaStreamSynchronize(st);
                    alpha.push_back(hcoef[j]);
                }
                count_launches(1);
                k_subtract<<<g, 256, 0, st>>>(dim, j + 1, V, coef, w);
            }
            // beta_j = |w|
            double *vn = V + (int64_t)(j + 1) * dim;
            count_launches(1);
            k_scale<<<g, 256, 0, st>>>(dim, w, 1.0, vn);
            {
                dim3 grid(kRedBlocks, 1);
                count_launches(1);
                k_multidot<<<grid, kRedThreads, 0, st>>>(dim, 1, vn, w, partial);
                count_launches(1);
                k_finish_dots<<<1, 32, 0, st>>>(1, kRedBlocks, partial, coef);
            }
            double b2 = 0.0;
            cudaMemcpyAsync(&b2, coef, sizeof(double), cudaMemcpyDeviceToHost, st);
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { rc = cuda_fail(e, "lanczos step"); break; }
            double bj = std::sqrt(std::max(b2, 0.0));
            beta.push_back(bj);
            m = j + 1;
            // Ritz values and residual bounds beta_j |last component|
            std::vector<double> d(alpha), off(beta.begin(), beta.end() - 1);
            if (off.empty()) off.push_back(0.0);
            tridiag_qr(m, d, off, Z);
            theta = d;
            int nv = std::min(nev, m);
            bool ok = m >= std::min<int64_t>(nev, dim);
            for (int r = 0; r < nv && ok; ++r) {
                double res = bj * std::fabs(Z[(size_t)(m - 1) * m + r]);
                if (res > tol * std::max(1.0, std::fabs(theta[r]))) ok = false;
            }
            bool invariant = bj <= 1e-12 * (std::fabs(alpha.back()) + 1.0);
            if (ok || invariant) { conv = true; break; }
            if (m == m_max) break;
            count_launches(1);
            k_scale<<<g, 256, 0, st>>>(dim, w, 1.0 / bj, vn);
        }
        if (rc) break;
        if (!conv) not_converged = 1;
        int nv = std::min(nev, m);
        for (int r = 0; r < nv; ++r) evals[(int64_t)set * nev + r] = theta[r];
        if (evec0) {
            for (int r = 0; r < m; ++r) hcoef[r] = Z[(size_t)r * m + 0];
            cudaMemcpyAsync(coef, hcoef.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st);
            double *out = evec0 + (int64_t)set * dim;
            count_launches(1);
            k_combine<<<g, 256, 0, st>>>(dim, m, V, coef, out);
            // normalise
            count_launches(1);
            k_scale<<<g, 256, 0, st>>>(dim, out, 1.0, w);
            dim3 grid(kRedBlocks, 1);
            count_launches(1);
            k_multidot<<<grid, kRedThreads, 0, st>>>(dim, 1, out, w, partial);
            count_launches(1);
            k_finish_dots<<<1, 32, 0, st>>>(1, kRedBlocks, partial, coef);
            double n2 = 1.0;
            cudaMemcpyAsync(&n2, coef, sizeof(double), cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);
            count_launches(1);
            k_scale<<<g, 256, 0, st>>>(dim, w, 1.0 / std::sqrt(n2), out);
        }
    }
    e = cudaGetLastError();
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "lanczos kernels");
    cudaFreeAsync(V, st);
    cudaFreeAsync(w, st);
    cudaFreeAsync(partial, st);
    cudaFreeAsync(coef, st);
    if (!rc) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "lanczos");
    }
    return rc ? rc : not_converged;
}

}  // namespace cih

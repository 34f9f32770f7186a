// Lanczos for the lowest eigenpairs (Sec. 2: successive matrix-vector
// products and orthogonalisations), for K matrices that share one half-stored
// structure, all K Krylov sequences advancing together.
//
// Device:
//   - the mirrored half of the symmetric matrix is read through a transposed
//     index of the strictly-upper part (for each column j, the stored (i, k)
//     with i < j, sorted by i), so y = H x needs no atomics and is
//     deterministic;
//   - values element-major (the K values of a nonzero together) and vectors
//     element-major x[i * K + s], FP64;
//   - full reorthogonalisation: classical Gram-Schmidt applied twice, dot
//     products reduced in two fixed-order stages.
// Host: per set (sets on parallel host threads), the lowest Ritz values and
// the residual bounds beta_m |z_m| from implicit-QR sweeps of the tridiagonal
// that rotate only the last row of its eigenvector matrix; the lowest Ritz
// vector's coefficients by inverse iteration.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "cih_internal.h"

namespace cih {
namespace {

// fn(s) for s = 0 .. K - 1, on up to 8 host threads when there is more than one set
template <class F>
void parallel_sets(int K, F &&fn)
{
    const int nt = std::min({K, 8, (int)std::max(1u, std::thread::hardware_concurrency())});
    if (nt <= 1) {
        for (int s = 0; s < K; ++s) fn(s);
        return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
            for (int s = t; s < K; s += nt) fn(s);
        });
    for (auto &x : th) x.join();
}

constexpr int kDotBlocks = 256;
constexpr int kThreads = 256;

// ---- transposed index of the strictly-upper part

__global__ void k_tcount(int64_t dim, const int64_t *rowptr, const int32_t *col, int32_t *tcnt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (col[k] != i) atomicAdd(&tcnt[col[k]], 1);
}

// entry of stored nonzero k = (i, j), i < j, in column j's list: (i << 32) |
// low, low = the value's bits when one set (the mirror pass then reads no
// other array), else k
__global__ void k_tfill(int64_t dim, const int64_t *rowptr, const int32_t *col, const int64_t *toff, int32_t *tcur,
                        const float *val1, int64_t *tent)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const int32_t j = col[k];
            if (j == i) continue;
            const int64_t at = toff[j] + atomicAdd(&tcur[j], 1);
            const uint32_t low = val1 ? __float_as_uint(val1[k]) : (uint32_t)k;
            tent[at] = (i << 32) | low;                      // sorts by row first
        }
}

// sort each column's entries by row (keys are distinct): bitonic in shared
// memory, for the columns with lo < length <= TILE
template <int TILE>
__global__ void k_tsort(int64_t dim, const int64_t *toff, int64_t *tent, int lo)
{
    extern __shared__ int64_t sh[];
    for (int64_t j = blockIdx.x; j < dim; j += gridDim.x) {
        const int64_t o = toff[j];
        const int64_t len64 = toff[j + 1] - o;
        if (len64 <= lo || len64 > TILE || len64 <= 1) continue;
        const int len = (int)len64;
        int P = 1;
        while (P < len) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) sh[i] = i < len ? tent[o + i] : INT64_MAX;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int s = k >> 1; s > 0; s >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    const int l = i ^ s;
                    if (l > i) {
                        const bool up = (i & k) == 0;
                        const int64_t a = sh[i], c = sh[l];
                        if ((a > c) == up) { sh[i] = c; sh[l] = a; }
                    }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < len; i += blockDim.x) tent[o + i] = sh[i];
        __syncthreads();
    }
}
constexpr int kTileSmall = 2048, kTileLarge = 16384;   // 16 KB and 128 KB of shared memory

// values of the transposed entries, element-major: vT[t * K + s] = vem[k(t) * K + s]
__global__ void k_vT(int64_t nt, int K, const int64_t *tent, const float *vem, float *vT)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nt * K; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = q / K;
        const int s = (int)(q - t * K);
        vT[q] = vem[(int64_t)(uint32_t)tent[t] * K + s];
    }
}

// element-major values: vem[k * K + s] = val[s * nnz + k]
__global__ void k_vals_em(int K, int64_t nnz, const float *val, float *vem)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz * K; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / K;
        const int s = (int)(t - k * K);
        vem[t] = val[(int64_t)s * nnz + k];
    }
}

// ---- y = H x for K sets.  One warp per row, row part then mirror part.
// K >= 32: lanes over sets, two sets per lane per pass, nonzeros four at a
// time; K < 32 (KS = next power of two): 32/KS lane groups split the
// nonzeros, four per group at a time, then reduce across the groups.  The
// four independent loads keep more of each row's gathers in flight.  The
// summation order depends only on the structure.
template <int KS>
__global__ void k_spmv(int64_t dim, int K, const int64_t *rowptr, const int32_t *col, const int64_t *toff,
                       const int64_t *tent, const float *vem, const float *vT, const double *x, double *y)
{
    const int lane = threadIdx.x & 31;
    // each block walks one contiguous run of rows, so that rows of the same
    // proton sub-determinant (which gather the same x blocks) share its L1
    const int64_t per = (dim + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * per, r1 = min(dim, r0 + per);
    const int wpb = blockDim.x >> 5;
    for (int64_t i = r0 + (threadIdx.x >> 5); i < r1; i += wpb) {
        const int64_t a0 = rowptr[i], a1 = rowptr[i + 1], b0 = toff[i], b1 = toff[i + 1];
        if (KS >= 32) {
            for (int s0 = 0; s0 < K; s0 += 64) {
                const int sa = s0 + lane, sb = s0 + 32 + lane;
                const bool ha = sa < K, hb = sb < K;
                double acc_a = 0.0, acc_b = 0.0;
                int64_t k = a0;
                for (; k + 3 < a1; k += 4) {
                    int64_t c[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) c[u] = (int64_t)col[k + u] * K;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (ha) acc_a += (double)vem[(k + u) * K + sa] * __ldg(x + c[u] + sa);
                        if (hb) acc_b += (double)vem[(k + u) * K + sb] * __ldg(x + c[u] + sb);
                    }
                }
                for (; k < a1; ++k) {
                    const int64_t c = (int64_t)col[k] * K;
                    if (ha) acc_a += (double)vem[k * K + sa] * __ldg(x + c + sa);
                    if (hb) acc_b += (double)vem[k * K + sb] * __ldg(x + c + sb);
                }
                int64_t t = b0;
                for (; t + 3 < b1; t += 4) {
                    int64_t r[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) r[u] = (tent[t + u] >> 32) * K;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (ha) acc_a += (double)vT[(t + u) * K + sa] * __ldg(x + r[u] + sa);
                        if (hb) acc_b += (double)vT[(t + u) * K + sb] * __ldg(x + r[u] + sb);
                    }
                }
                for (; t < b1; ++t) {
                    const int64_t r = (tent[t] >> 32) * K;
                    if (ha) acc_a += (double)vT[t * K + sa] * __ldg(x + r + sa);
                    if (hb) acc_b += (double)vT[t * K + sb] * __ldg(x + r + sb);
                }
                if (ha) y[i * K + sa] = acc_a;
                if (hb) y[i * K + sb] = acc_b;
            }
        } else {
            constexpr int G = 32 / KS;
            const int g = lane / KS, s = lane % KS;
            double acc = 0.0;
            if (s < K) {
                int64_t k = a0 + g;
                for (; k + 3 * G < a1; k += 4 * G) {
                    int64_t c[4];
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        c[u] = col[k + u * G];
                        v[u] = vem[(k + u * G) * K + s];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) acc += (double)v[u] * __ldg(x + c[u] * K + s);
                }
                for (; k < a1; k += G) acc += (double)vem[k * K + s] * __ldg(x + (int64_t)col[k] * K + s);
                int64_t t = b0 + g;
                for (; t + 3 * G < b1; t += 4 * G) {
                    int64_t e[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) e[u] = tent[t + u * G];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float v = KS == 1 ? __uint_as_float((uint32_t)e[u]) : vT[(t + u * G) * K + s];
                        acc += (double)v * __ldg(x + (e[u] >> 32) * K + s);
                    }
                }
                for (; t < b1; t += G) {
                    const int64_t e = tent[t];
                    const float v = KS == 1 ? __uint_as_float((uint32_t)e) : vT[t * K + s];
                    acc += (double)v * __ldg(x + (e >> 32) * K + s);
                }
            }
            for (int d = 16; d >= KS; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
            if (g == 0 && s < K) y[i * K + s] = acc;
        }
    }
}

// partial[(r * K + s) * gridDim.x + blk] = sum over this block's rows of V[r][i][s] w[i][s]
__global__ void k_dots(int64_t dim, int K, int nvec, const double *V, int64_t vstride, const double *w,
                       double *partial)
{
    __shared__ double red[kThreads];
    const int per = kThreads / K;                    // rows per pass (K <= kThreads)
    const int s = threadIdx.x % K, sub = threadIdx.x / K;
    const bool act = sub < per;
    for (int r = blockIdx.y; r < nvec; r += gridDim.y) {
        const double *v = V + (int64_t)r * vstride;
        double acc = 0.0;
        if (act)
            for (int64_t i = (int64_t)blockIdx.x * per + sub; i < dim; i += (int64_t)gridDim.x * per)
                acc += v[i * K + s] * w[i * K + s];
        red[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x < K) {
            double t = 0.0;
            for (int q = 0; q < per; ++q) t += red[q * K + threadIdx.x];
            partial[((int64_t)r * K + threadIdx.x) * gridDim.x + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

// out[q] = fixed-order sum of the partials of q = r * K + s
__global__ void k_dots_finish(int n, int parts, const double *partial, double *out)
{
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int b = 0; b < parts; ++b) t += partial[(int64_t)q * parts + b];
        out[q] = t;
    }
}

// w[i][s] -= sum_r h[r][s] V[r][i][s]
__global__ void k_subtract(int64_t n, int K, int nvec, const double *V, int64_t vstride, const double *h, double *w)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(t % K);
        double acc = w[t];
        for (int r = 0; r < nvec; ++r) acc -= h[r * K + s] * V[(int64_t)r * vstride + t];
        w[t] = acc;
    }
}

// out[t] = in[t] * f[s]
__global__ void k_scale_sets(int64_t n, int K, const double *in, const double *f, double *out)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = in[t] * f[t % K];
}

// deterministic start vector: 1 + 0.5 u_i, u_i from the splitmix64 hash of i (same for every set)
__global__ void k_start(int64_t dim, int K, double *v)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * K; t += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long z = (unsigned long long)(t / K) + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        v[t] = 1.0 + 0.5 * (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
}

// evec[s * dim + i] = sum_r c[r * K + s] V[r][i][s]  (set-major output)
__global__ void k_ritz(int64_t dim, int K, int m, const double *V, int64_t vstride, const double *c, double *evec)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < dim * K; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / K;
        const int s = (int)(t - i * K);
        double acc = 0.0;
        for (int r = 0; r < m; ++r) acc += c[r * K + s] * V[(int64_t)r * vstride + t];
        evec[(int64_t)s * dim + i] = acc;
    }
}

// normalise each set-major vector: block s reduces set s in a fixed order
__global__ void k_normalise_sets(int64_t dim, double *evec)
{
    __shared__ double red[kThreads];
    double *v = evec + (int64_t)blockIdx.x * dim;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < dim; i += blockDim.x) acc += v[i] * v[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int d = kThreads / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
        __syncthreads();
    }
    const double f = red[0] > 0.0 ? 1.0 / sqrt(red[0]) : 0.0;
    for (int64_t i = threadIdx.x; i < dim; i += blockDim.x) v[i] *= f;
}

int grid_for(int64_t n)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 16));
}

}  // namespace

int64_t lanczos_bytes(int64_t dim, int64_t nnz, int K, int max_iter)
{
    const int64_t m = std::min<int64_t>(max_iter, dim);
    const int64_t nt = std::max<int64_t>(nnz - dim, 1);
    int64_t bytes = 4 * (dim + 1) + 8 * (dim + 1) + 8 * nt;          // transposed index
    bytes += 8 * (m + 1) * dim * K + 8 * dim * K;                   // Lanczos vectors, w
    bytes += 8 * (m + 1) * K * kDotBlocks + 8 * (m + 1) * K + 8 * K; // dot partials, h, scale
    if (K > 1) bytes += 4 * nnz * K + 4 * nt * K;                   // element-major values, mirror values
    return bytes + 8 * 256;                                         // allocation granules
}

int lanczos(const cih_basis &b, const int64_t *rowptr, const int32_t *col, const float *val, int K, int nev,
            int max_iter, double tol, double *evals, double *evec0, cudaStream_t st, bool values_em)
{
    const int64_t dim = b.dim;
    for (int k = 0; k < K * nev; ++k) evals[k] = NAN;
    if (dim == 0) return CIH_OK;
    if (K > kThreads) return fail(CIH_ERR_UNSUPPORTED, "lanczos: at most 256 sets per call");
    if (dim > INT32_MAX) return fail(CIH_ERR_UNSUPPORTED, "lanczos: dimension above 2^31");
    int64_t nnz = 0;
    cudaError_t e = cudaMemcpyAsync(&nnz, rowptr + dim, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "lanczos: read nnz");
    const int m_max = (int)std::min<int64_t>(max_iter, dim);
    const int64_t vstride = dim * K;

    std::vector<void *> bufs;
    auto alloc = [&](void **p, size_t bytes) -> bool {
        if (cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), b.pool, st) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        bufs.push_back(*p);
        return true;
    };
    int32_t *tcnt = nullptr;
    int64_t *toff = nullptr, *tent = nullptr;
    float *vem = nullptr, *vT = nullptr;
    double *V = nullptr, *w = nullptr, *partial = nullptr, *hdev = nullptr, *fdev = nullptr;
    const int64_t nt = std::max<int64_t>(nnz - dim, 1);             // strictly upper entries
    bool ok = alloc((void **)&tcnt, sizeof(int32_t) * (dim + 1)) && alloc((void **)&toff, sizeof(int64_t) * (dim + 1)) &&
              alloc((void **)&tent, sizeof(int64_t) * nt) &&
              alloc((void **)&V, sizeof(double) * (size_t)(m_max + 1) * vstride) &&
              alloc((void **)&w, sizeof(double) * vstride) &&
              alloc((void **)&partial, sizeof(double) * (size_t)(m_max + 1) * K * kDotBlocks) &&
              alloc((void **)&hdev, sizeof(double) * (size_t)(m_max + 1) * K) && alloc((void **)&fdev, sizeof(double) * K);
    if (ok && K > 1 && !values_em) ok = alloc((void **)&vem, sizeof(float) * (size_t)nnz * K);
    if (ok && K > 1) ok = alloc((void **)&vT, sizeof(float) * (size_t)nt * K);
    int rc = ok ? CIH_OK : fail(CIH_ERR_NOMEM, "lanczos: device memory");
    const int g = grid_for(vstride);
    const int gr = (int)std::min<int64_t>((dim + 7) / 8, 152 * 32);

    // transposed index (built once for all sets)
    if (!rc) {
        cudaMemsetAsync(tcnt, 0, sizeof(int32_t) * (dim + 1), st);
        count_launches(1);
        k_tcount<<<grid_for(dim), kThreads, 0, st>>>(dim, rowptr, col, tcnt);
        std::vector<int32_t> hc(dim);
        e = cudaMemcpyAsync(hc.data(), tcnt, sizeof(int32_t) * dim, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "lanczos: transpose count");
        if (!rc) {
            std::vector<int64_t> ho(dim + 1, 0);
            for (int64_t j = 0; j < dim; ++j) ho[j + 1] = ho[j] + hc[j];
            cudaMemcpyAsync(toff, ho.data(), sizeof(int64_t) * (dim + 1), cudaMemcpyHostToDevice, st);
            cudaMemsetAsync(tcnt, 0, sizeof(int32_t) * (dim + 1), st);
            count_launches(1);
            k_tfill<<<grid_for(dim), kThreads, 0, st>>>(dim, rowptr, col, toff, tcnt, K == 1 ? val : nullptr, tent);
            // columns up to 2048 entries, then the longer ones (up to 16384) one per SM;
            // longer columns keep the fill order, which may vary from run to run
            const int gs = (int)std::min<int64_t>(dim, 65535);
            count_launches(2);
            k_tsort<kTileSmall><<<gs, 256, kTileSmall * sizeof(int64_t), st>>>(dim, toff, tent, 1);
            cudaFuncSetAttribute(k_tsort<kTileLarge>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kTileLarge * (int)sizeof(int64_t));
            k_tsort<kTileLarge><<<152, 1024, kTileLarge * sizeof(int64_t), st>>>(dim, toff, tent, kTileSmall);
            if (K > 1 && !values_em) {
                count_launches(1);
                k_vals_em<<<grid_for(nnz * K), kThreads, 0, st>>>(K, nnz, val, vem);
            } else {
                vem = const_cast<float *>(val);                     // already element-major
            }
            if (K > 1 && nnz > dim) {                               // mirror values in column order
                count_launches(1);
                k_vT<<<grid_for((nnz - dim) * K), kThreads, 0, st>>>(nnz - dim, K, tent, vem, vT);
            }
            e = cudaStreamSynchronize(st);                          // the host offsets go out of scope here
            if (e != cudaSuccess) rc = cuda_fail(e, "lanczos: transpose");
        }
    }

    auto spmv = [&](const double *x, double *y) {
        count_launches(1);
        if (K >= 32) k_spmv<32><<<gr, kThreads, 0, st>>>(dim, K, rowptr, col, toff, tent, vem, vT, x, y);
        else if (K == 1) k_spmv<1><<<gr, kThreads, 0, st>>>(dim, K, rowptr, col, toff, tent, vem, vT, x, y);
        else if (K <= 2) k_spmv<2><<<gr, kThreads, 0, st>>>(dim, K, rowptr, col, toff, tent, vem, vT, x, y);
        else if (K <= 4) k_spmv<4><<<gr, kThreads, 0, st>>>(dim, K, rowptr, col, toff, tent, vem, vT, x, y);
        else if (K <= 8) k_spmv<8><<<gr, kThreads, 0, st>>>(dim, K, rowptr, col, toff, tent, vem, vT, x, y);
        else k_spmv<16><<<gr, kThreads, 0, st>>>(dim, K, rowptr, col, toff, tent, vem, vT, x, y);
    };
    // h[r][s] = V[r] . w for r < nvec: into hdev (device) and hh (host)
    std::vector<double> hh((size_t)(m_max + 1) * K);
    auto dots = [&](const double *vb, int nvec, const double *wv) -> int {
        dim3 grid(kDotBlocks, std::min(nvec, 65535));
        count_launches(2);
        k_dots<<<grid, kThreads, 0, st>>>(dim, K, nvec, vb, vstride, wv, partial);
        k_dots_finish<<<(nvec * K + 255) / 256, 256, 0, st>>>(nvec * K, kDotBlocks, partial, hdev);
        cudaError_t ee = cudaMemcpyAsync(hh.data(), hdev, sizeof(double) * nvec * K, cudaMemcpyDeviceToHost, st);
        if (ee == cudaSuccess) ee = cudaStreamSynchronize(st);
        return ee == cudaSuccess ? CIH_OK : cuda_fail(ee, "lanczos: dots");
    };
    std::vector<double> fh(K);
    auto scale = [&](const double *in, double *out) {
        cudaMemcpyAsync(fdev, fh.data(), sizeof(double) * K, cudaMemcpyHostToDevice, st);
        count_launches(1);
        k_scale_sets<<<g, kThreads, 0, st>>>(vstride, K, in, fdev, out);
    };

    // v0 = start / |start| per set
    if (!rc) {
        count_launches(1);
        k_start<<<g, kThreads, 0, st>>>(dim, K, w);
        rc = dots(w, 1, w);
        for (int s = 0; s < K && !rc; ++s) fh[s] = 1.0 / std::sqrt(hh[s]);
        if (!rc) scale(w, V);
    }
    std::vector<std::vector<double>> alpha(K), beta(K);
    std::vector<int> done(K, 0), m_of(K, 0), met(K, 0);
    std::vector<double> theta((size_t)K * nev, NAN);
    int m = 0;
    for (int j = 0; j < m_max && !rc; ++j) {
        spmv(V + (int64_t)j * vstride, w);
        for (int pass = 0; pass < 2 && !rc; ++pass) {
            if ((rc = dots(V, j + 1, w))) break;
            for (int s = 0; s < K; ++s)                             // alpha_j = v_j . H v_j (+ the
                if (!done[s]) {                                     // second pass's small correction)
                    if (pass == 0) alpha[s].push_back(hh[(size_t)j * K + s]);
                    else alpha[s].back() += hh[(size_t)j * K + s];
                }
            count_launches(1);
            k_subtract<<<g, kThreads, 0, st>>>(vstride, K, j + 1, V, vstride, hdev, w);
        }
        if (rc || (rc = dots(w, 1, w))) break;
        m = j + 1;
        // per set (sets in parallel on host threads): Ritz values and residual
        // bounds beta_m |z_m| of the lowest nev, from the tridiagonal's QR
        // eigen-decomposition (last eigenvector components)
        parallel_sets(K, [&](int s) {
            fh[s] = 0.0;
            if (done[s]) return;
            const double bj = std::sqrt(std::max(hh[s], 0.0));
            beta[s].push_back(bj);
            const int ms = m_of[s] = (int)alpha[s].size();
            const int nv = std::min(nev, ms);
            bool conv = ms >= std::min<int64_t>(nev, dim);
            const bool invariant = bj <= 1e-12 * (std::fabs(alpha[s].back()) + 1.0);
            std::vector<double> dq(alpha[s]), eq(beta[s].begin(), beta[s].begin() + (ms - 1)), zl;
            if (eq.empty()) eq.push_back(0.0);
            tridiag_qr_last(ms, dq, eq, zl);
            for (int r = 0; r < nv; ++r) {
                const double th = dq[r];
                theta[(size_t)s * nev + r] = th;
                if (conv && !invariant && bj * std::fabs(zl[r]) > tol * std::max(1.0, std::fabs(th))) conv = false;
            }
            met[s] = conv || invariant;
            if (met[s] || ms == m_max) done[s] = 1;
            else fh[s] = 1.0 / bj;                                  // next vector; frozen sets get zeros
        });
        bool all = true;
        for (int s = 0; s < K; ++s) all = all && done[s];
        if (all) break;
        scale(w, V + (int64_t)(j + 1) * vstride);
    }
    int not_converged = 0;
    if (!rc) {
        std::vector<double> coef((size_t)std::max(m, 1) * K, 0.0);
        for (int s = 0; s < K; ++s) {
            const int ms = m_of[s];
            for (int r = 0; r < std::min(nev, ms); ++r) evals[(int64_t)s * nev + r] = theta[(size_t)s * nev + r];
            if (!met[s]) not_converged = 1;
            if (evec0 && ms > 0) {
                std::vector<double> z(ms);
                tridiag_eigenvector(ms, alpha[s].data(), beta[s].data(), theta[(size_t)s * nev], z.data());
                for (int r = 0; r < ms; ++r) coef[(size_t)r * K + s] = z[r];
            }
        }
        if (evec0 && m > 0) {
            cudaMemcpyAsync(hdev, coef.data(), sizeof(double) * (size_t)m * K, cudaMemcpyHostToDevice, st);
            count_launches(2);
            k_ritz<<<g, kThreads, 0, st>>>(dim, K, m, V, vstride, hdev, evec0);
            k_normalise_sets<<<K, kThreads, 0, st>>>(dim, evec0);
        }
    }
    e = cudaGetLastError();
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "lanczos kernels");
    for (void *p : bufs) cudaFreeAsync(p, st);
    if (!rc) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "lanczos");
    }
    cudaMemPoolTrimTo(b.pool, 0);                            // the Lanczos vectors go back to the system
    return rc ? rc : not_converged;
}

}  // namespace cih

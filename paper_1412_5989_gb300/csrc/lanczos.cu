// Lanczos for the lowest eigenpairs (Sec. 2: successive matrix-vector
// products and orthogonalisations), for K matrices that share one half-stored
// structure, all K Krylov sequences advancing together.
//
// Device:
//   - y = H x reads each stored nonzero of the upper half once: the row part
//     as double-float sums of FP32-pair products, the mirrored half added to
//     64-bit fixed-point column accumulators (integer atomic adds commute, so
//     y is deterministic); no FP64 operation per nonzero;
//   - over row shards held by several processes, each multiplies its own rows
//     and a caller callback sums the two product buffers across them;
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
#include "ham_common.cuh"

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

// element-major values: vem[k * K + s] = val[s * nnz + k]
__global__ void k_vals_em(int K, int64_t nnz, const float *val, float *vem)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz * K; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / K;
        const int s = (int)(t - k * K);
        vem[t] = val[(int64_t)s * nnz + k];
    }
}

// Rows [r0, r1) of the matrix whose column and value arrays start at stored
// nonzero `base` (0 for a whole matrix; rowptr[r0] for a row shard).
struct RowRange {
    int64_t r0, r1, base;
};

// ---- y = H x from the stored upper half, each stored nonzero read once.
//
// Row i's warp forms the row part sum_j h_ij x_j (double-float sums in a
// fixed order: lanes, then a shuffle tree), and sends each strictly-upper h_ij x_i
// to column j's accumulator as a 64-bit fixed-point integer (units 2^-s) by
// an atomic add.  Integer adds commute, so y does not depend on the order in
// which rows run: the product is deterministic without a transposed copy.
// k_sym_finish adds the two parts and clears the accumulators.
//
// The scale 2^s keeps every accumulator inside 2^60: for column j,
// |sum_{i<j} h_ij x_i| <= ||h_{.j}|| ||x|| (Cauchy-Schwarz) <= F ||x||, with
// F the Frobenius norm of the strictly-upper part over all sets, and the
// Lanczos vectors have ||x|| = 1.  Each product, an FP32 pair, enters as its
// rounded hi plus its rounded lo: at most one unit 2^-s of absolute error.

// partial[blk] = this block's sum of the squares of the strictly-upper
// values of all sets (a warp per row, lanes over (nonzero, set) pairs), in
// double-float sums of the exact FP32-pair squares
constexpr int kSumsqThreads = 1024;
__global__ void __launch_bounds__(kSumsqThreads) k_upper_sumsq(RowRange rr, int K, const int64_t *rowptr,
                                                               const float *vem, double *partial)
{
    __shared__ double red[kSumsqThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    DF acc = df_of(0.f);
    for (int64_t i = rr.r0 + blockIdx.x * (int64_t)(blockDim.x >> 5) + wid; i < rr.r1;
         i += (int64_t)gridDim.x * (blockDim.x >> 5)) {
        const int64_t t1 = (rowptr[i + 1] - rr.base) * K;
#pragma unroll 4
        for (int64_t t = (rowptr[i] - rr.base + 1) * K + lane; t < t1; t += 32) {
            const float v = vem[t];
            const float p = v * v;
            acc = df_add(acc, DF{p, fmaf(v, v, -p)});
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        const DF o{__shfl_xor_sync(0xffffffffu, acc.hi, d), __shfl_xor_sync(0xffffffffu, acc.lo, d)};
        acc = df_add(acc, o);
    }
    if (lane == 0) red[wid] = (double)acc.hi + (double)acc.lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// sc = (2^s, 2^-s, 2^r, 2^-r) from the sum of squares F^2 (fixed-order sum
// of the partials) and, when given, the largest squared norm of the K
// vectors (else the vectors have norm 1), with F ||x|| < 2^e and ||x|| < 2^ex:
//   s = min(60 - e, 124 - ex): the mirrored products' units 2^-s keep every
//       accumulator below 2^60, and every x_i 2^s is an FP32 pair;
//   r = 1 - ex: the row part multiplies x 2^r, of norm below 2 (0 when the
//       vectors have norm 1).
__global__ void k_mirror_scale(int parts, const double *partial, int K, const double *xn2, double *sc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double f2 = 0.0;
    for (int b = 0; b < parts; ++b) f2 += partial[b];
    double m = 1.0;
    if (xn2) {
        m = 0.0;
        for (int k = 0; k < K; ++k) m = fmax(m, xn2[k]);
    }
    int e = 0, ex = 1;
    if (f2 > 0.0 && m > 0.0) (void)frexp(sqrt(f2 * m) * (1.0 + 1e-6), &e);
    if (xn2 && m > 0.0) (void)frexp(sqrt(m) * (1.0 + 1e-6), &ex);
    const int sh = min(60 - e, 124 - ex), r = xn2 ? 1 - ex : 0;
    sc[0] = ldexp(1.0, sh);
    sc[1] = ldexp(1.0, -sh);
    sc[2] = ldexp(1.0, r);
    sc[3] = ldexp(1.0, -r);
}

// The GPU's FP64 units are few, so the product runs in FP32 pairs: x is
// split once per product into hi + lo floats (xs), a product v (hi + lo) is
// the pair (v hi, fma(v, hi, -v hi) + v lo) (about 47 bits), row sums are
// double-float sums, and a mirrored product goes to the fixed-point
// accumulator as the rounded hi plus the rounded lo (at most 1 unit of
// error).  No FP64 operation runs per stored nonzero.
__device__ __forceinline__ float2 split2(double v)
{
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

__device__ __forceinline__ DF df_prod(float v, float2 x)
{
    const float p = v * x.x;
    return DF{p, fmaf(v, x.y, fmaf(v, x.x, -p))};
}

// f rounded to the nearest integer (halves away from zero) by integer
// operations on its bits; |f| < 2^62.  (The hardware's 64-bit conversions run
// on the FP64 units.)
__device__ __forceinline__ long long round_ll(float f)
{
    const unsigned b = __float_as_uint(f);
    const int sh = (int)((b >> 23) & 0xFFu) - 150;                 // |f| = m 2^sh
    const unsigned m = (b & 0x7FFFFFu) | 0x800000u;
    long long v = 0;                                                // |f| < 0.5, zero, subnormal
    if (sh >= 0) v = (long long)m << sh;
    else if (sh >= -24) v = (long long)((m + (1u << (-sh - 1))) >> -sh);
    return (b >> 31) ? -v : v;
}

__device__ __forceinline__ void mirror_add(unsigned long long *a, DF q)
{
    atomicAdd(a, (unsigned long long)(round_ll(q.hi) + round_ll(q.lo)));
}

// xs[t] = x[t] 2^r (the row part's factor) and xm[t] = x[t] 2^s (the
// mirrored products'), each as hi + lo floats
__global__ void k_split(int64_t n, const double *x, const double *sc, float2 *xs, float2 *xm)
{
    const double fr = sc[2], fs = sc[0];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[t];
        xs[t] = split2(v * fr);
        xm[t] = split2(v * fs);
    }
}

// K >= 32: lanes over sets, two per lane per pass; K < 32 (KS = next power
// of two): 32/KS lane groups split the row's nonzeros, four at a time per
// group, and the groups' row sums are reduced at the end.  With K < 32 the
// matrix is read with evict-first loads, so that its stream does not push x
// and the accumulators out of L2 (with lanes over sets the same hint ran
// slower).  Each block walks
// one contiguous run of rows, so that rows of one proton sub-determinant
// (which touch the same x and accumulator blocks) share its L1.
template <int KS>
__global__ void __launch_bounds__(kThreads, 4) k_spmv(RowRange rr, int K, const int64_t *rowptr, const int32_t *col, const float *vem,
                       const float2 *xs, const float2 *xm, float2 *yrow, unsigned long long *yfix)
{
    const int lane = threadIdx.x & 31;
    const int64_t per = (rr.r1 - rr.r0 + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = rr.r0 + blockIdx.x * per, r1 = min(rr.r1, r0 + per);
    const int wpb = blockDim.x >> 5;
    for (int64_t i = r0 + (threadIdx.x >> 5); i < r1; i += wpb) {
        const int64_t a0 = rowptr[i] - rr.base, a1 = rowptr[i + 1] - rr.base;
        if (KS >= 32) {
            const int KK = KS == 64 ? 64 : K;                      // KS = 64: exactly 64 sets
            for (int s0 = 0; s0 < KK; s0 += 64) {
                const int sa = s0 + lane, sb = s0 + 32 + lane;
                const bool ha = sa < KK, hb = sb < KK;
                const float2 Xa = ha ? xm[i * KK + sa] : make_float2(0.f, 0.f);
                const float2 Xb = hb ? xm[i * KK + sb] : make_float2(0.f, 0.f);
                DF acc_a = df_of(0.f), acc_b = df_of(0.f);
                int64_t k = a0;
                for (; k + 3 < a1; k += 4) {
                    int64_t c[4];
                    float va[4], vb[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        c[u] = col[k + u];
                        va[u] = ha ? vem[(k + u) * KK + sa] : 0.f;
                        vb[u] = hb ? vem[(k + u) * KK + sb] : 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (ha) acc_a = df_add(acc_a, df_prod(va[u], xs[c[u] * KK + sa]));
                        if (hb) acc_b = df_add(acc_b, df_prod(vb[u], xs[c[u] * KK + sb]));
                        if (c[u] != i) {
                            if (ha) mirror_add(yfix + c[u] * KK + sa, df_prod(va[u], Xa));
                            if (hb) mirror_add(yfix + c[u] * KK + sb, df_prod(vb[u], Xb));
                        }
                    }
                }
                for (; k < a1; ++k) {
                    const int64_t c = col[k];
                    const float va = ha ? vem[k * KK + sa] : 0.f, vb = hb ? vem[k * KK + sb] : 0.f;
                    if (ha) acc_a = df_add(acc_a, df_prod(va, xs[c * KK + sa]));
                    if (hb) acc_b = df_add(acc_b, df_prod(vb, xs[c * KK + sb]));
                    if (c != i) {
                        if (ha) mirror_add(yfix + c * KK + sa, df_prod(va, Xa));
                        if (hb) mirror_add(yfix + c * KK + sb, df_prod(vb, Xb));
                    }
                }
                if (ha) yrow[i * KK + sa] = make_float2(acc_a.hi, acc_a.lo);
                if (hb) yrow[i * KK + sb] = make_float2(acc_b.hi, acc_b.lo);
            }
        } else {
            constexpr int G = 32 / KS;
            const int g = lane / KS, s = lane % KS;
            DF acc = df_of(0.f);
            if (s < K) {
                const float2 Xi = xm[i * K + s];
                int64_t k = a0 + g;
                for (; k + 3 * G < a1; k += 4 * G) {
                    int64_t c[4];
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        c[u] = __ldcs(col + k + u * G);
                        v[u] = __ldcs(vem + (k + u * G) * K + s);
                    }
                    float2 xj[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) xj[u] = xs[c[u] * K + s];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        acc = df_add(acc, df_prod(v[u], xj[u]));
                        if (c[u] != i) mirror_add(yfix + c[u] * K + s, df_prod(v[u], Xi));
                    }
                }
                for (; k < a1; k += G) {
                    const int64_t c = __ldcs(col + k);
                    const float v = __ldcs(vem + k * K + s);
                    acc = df_add(acc, df_prod(v, xs[c * K + s]));
                    if (c != i) mirror_add(yfix + c * K + s, df_prod(v, Xi));
                }
            }
            for (int d = 16; d >= KS; d >>= 1) {
                const DF o{__shfl_xor_sync(0xffffffffu, acc.hi, d), __shfl_xor_sync(0xffffffffu, acc.lo, d)};
                acc = df_add(acc, o);
            }
            if (g == 0 && s < K) yrow[i * K + s] = make_float2(acc.hi, acc.lo);
        }
    }
}

// y[t] = row part 2^-r + mirrored part 2^-s; the accumulators are cleared
// for the next product
__global__ void k_sym_finish(int64_t n, const double *sc, const float2 *yrow, double *y, unsigned long long *yfix)
{
    const double sinv = sc[1], rinv = sc[3];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float2 r = yrow[t];
        y[t] = ((double)r.x + (double)r.y) * rinv + (double)(long long)yfix[t] * sinv;
        yfix[t] = 0ull;
    }
}

// Row shards: the local rows' row part in FP64 into yx (the other entries
// stay 0, so that a sum over the shards is exact); then, once the caller has
// summed yx and the accumulators over the shards, y = yx + acc 2^-s and both
// are cleared.  The same operations in the same order as k_sym_finish.
__global__ void k_shard_rows(RowRange rr, int K, const double *sc, const float2 *yrow, double *yx)
{
    const double rinv = sc[3];
    const int64_t n = (rr.r1 - rr.r0) * K, o = rr.r0 * K;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const float2 r = yrow[o + t];
        yx[o + t] = ((double)r.x + (double)r.y) * rinv;
    }
}

__global__ void k_shard_finish(int64_t n, const double *sc, double *yx, unsigned long long *acc, double *y)
{
    const double sinv = sc[1];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        y[t] = yx[t] + (double)(long long)acc[t] * sinv;
        yx[t] = 0.0;
        acc[t] = 0ull;
    }
}

// One product's k_spmv launch.  (Passes of 32 sets, to keep a share of the
// randomly accessed vectors L2-resident at 64 sets, ran slower.)
void launch_spmv(RowRange rr, int K, const int64_t *rowptr, const int32_t *col, const float *vem, const float2 *xs,
                 const float2 *xm, float2 *yrow, unsigned long long *yfix, int gr, cudaStream_t st)
{
    count_launches(1);
    if (K == 64) k_spmv<64><<<gr, kThreads, 0, st>>>(rr, K, rowptr, col, vem, xs, xm, yrow, yfix);
    else if (K >= 32) k_spmv<32><<<gr, kThreads, 0, st>>>(rr, K, rowptr, col, vem, xs, xm, yrow, yfix);
    else if (K == 1) k_spmv<1><<<gr, kThreads, 0, st>>>(rr, K, rowptr, col, vem, xs, xm, yrow, yfix);
    else if (K <= 2) k_spmv<2><<<gr, kThreads, 0, st>>>(rr, K, rowptr, col, vem, xs, xm, yrow, yfix);
    else if (K <= 4) k_spmv<4><<<gr, kThreads, 0, st>>>(rr, K, rowptr, col, vem, xs, xm, yrow, yfix);
    else if (K <= 8) k_spmv<8><<<gr, kThreads, 0, st>>>(rr, K, rowptr, col, vem, xs, xm, yrow, yfix);
    else k_spmv<16><<<gr, kThreads, 0, st>>>(rr, K, rowptr, col, vem, xs, xm, yrow, yfix);
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
    int64_t bytes = 8 * (m + 1) * dim * K + 8 * dim * K;            // Lanczos vectors, w
    bytes += 32 * dim * K;                                          // mirror accumulators, split x, row part
    bytes += 8 * (m + 1) * K * kDotBlocks + 8 * (m + 1) * K + 8 * K + 32; // dot partials, h, scale
    if (K > 1) bytes += 4 * nnz * K;                                // element-major values
    return bytes + 8 * 256;                                         // allocation granules
}

// sh->f2 -> (2^s, 2^-s, 1, 1): the scale k_mirror_scale gives unit vectors
static void shard_scale(double f2, double *sc)
{
    int e = 0;
    if (f2 > 0.0) (void)std::frexp(std::sqrt(f2) * (1.0 + 1e-6), &e);
    const int sh = std::min(60 - e, 124 - 1);
    sc[0] = std::ldexp(1.0, sh);
    sc[1] = std::ldexp(1.0, -sh);
    sc[2] = sc[3] = 1.0;
}

int lanczos(const cih_basis &b, const int64_t *rowptr, const int32_t *col, const float *val, int K, int nev,
            int max_iter, double tol, double *evals, double *evec0, cudaStream_t st, bool values_em,
            const ShardRun *sh)
{
    const int64_t dim = b.dim;
    for (int k = 0; k < K * nev; ++k) evals[k] = NAN;
    if (dim == 0) return CIH_OK;
    if (K > kThreads) return fail(CIH_ERR_UNSUPPORTED, "lanczos: at most 256 sets per call");
    if (dim > INT32_MAX) return fail(CIH_ERR_UNSUPPORTED, "lanczos: dimension above 2^31");
    // the rows this process multiplies, and the stored nonzeros its arrays hold
    const int64_t r0 = sh ? sh->r0 : 0, r1 = sh ? sh->r1 : dim;
    int64_t ends[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&ends[0], rowptr + r0, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], rowptr + r1, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "lanczos: read nnz");
    const int64_t base = sh ? ends[0] : 0, nnz = ends[1] - base;
    const RowRange rr{r0, r1, base};
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
    float *vem = nullptr;
    unsigned long long *yfix = nullptr;
    float2 *xs = nullptr, *xm = nullptr, *yrow = nullptr;
    double *V = nullptr, *w = nullptr, *partial = nullptr, *hdev = nullptr, *fdev = nullptr, *sc = nullptr;
    bool ok = (sh ? (yfix = sh->acc) != nullptr : alloc((void **)&yfix, sizeof(unsigned long long) * (size_t)vstride)) &&
              alloc((void **)&xs, sizeof(float2) * (size_t)vstride) &&
              alloc((void **)&xm, sizeof(float2) * (size_t)vstride) &&
              alloc((void **)&yrow, sizeof(float2) * (size_t)vstride) &&
              alloc((void **)&V, sizeof(double) * (size_t)(m_max + 1) * vstride) &&
              alloc((void **)&w, sizeof(double) * vstride) &&
              alloc((void **)&partial, sizeof(double) * (size_t)(m_max + 1) * K * kDotBlocks) &&
              alloc((void **)&hdev, sizeof(double) * (size_t)(m_max + 1) * K) && alloc((void **)&fdev, sizeof(double) * K) &&
              alloc((void **)&sc, sizeof(double) * 4);
    if (ok && K > 1 && !values_em) ok = alloc((void **)&vem, sizeof(float) * (size_t)nnz * K);
    int rc = ok ? CIH_OK : fail(CIH_ERR_NOMEM, "lanczos: device memory");
    const int g = grid_for(vstride);
    const int gr = (int)std::max<int64_t>(1, std::min<int64_t>((r1 - r0 + 7) / 8, 152 * 32));

    // element-major values, the mirror scale and cleared accumulators (no host
    // synchronisation; a shard's scale comes from the whole matrix's norm)
    if (!rc) {
        if (K > 1 && !values_em) {
            count_launches(1);
            k_vals_em<<<grid_for(nnz * K), kThreads, 0, st>>>(K, nnz, val, vem);
        } else {
            vem = const_cast<float *>(val);                         // K = 1, or already element-major
        }
        if (sh) {
            double hsc[4];
            shard_scale(sh->f2, hsc);
            e = cudaMemcpyAsync(sc, hsc, sizeof(hsc), cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = cuda_fail(e, "lanczos: shard scale");
        } else {
            cudaMemsetAsync(yfix, 0, sizeof(unsigned long long) * (size_t)vstride, st);
            count_launches(2);
            k_upper_sumsq<<<kDotBlocks, kSumsqThreads, 0, st>>>(rr, K, rowptr, vem, partial);
            k_mirror_scale<<<1, 32, 0, st>>>(kDotBlocks, partial, K, nullptr, sc);
        }
    }

    auto spmv = [&](const double *x, double *y) -> int {
        count_launches(2);
        k_split<<<g, kThreads, 0, st>>>(vstride, x, sc, xs, xm);
        launch_spmv(rr, K, rowptr, col, vem, xs, xm, yrow, yfix, gr, st);
        if (!sh) {
            k_sym_finish<<<g, kThreads, 0, st>>>(vstride, sc, yrow, y, yfix);
            return CIH_OK;
        }
        // a shard: its rows' row part, then the caller sums both buffers over the shards
        count_launches(2);
        k_shard_rows<<<grid_for((r1 - r0) * K), kThreads, 0, st>>>(rr, K, sc, yrow, sh->yx);
        cudaError_t ee = cudaStreamSynchronize(st);
        if (ee != cudaSuccess) return cuda_fail(ee, "lanczos: shard product");
        if (sh->combine(sh->ctx) != 0) return fail(CIH_ERR_ARG, "lanczos: the shard combine callback failed");
        k_shard_finish<<<g, kThreads, 0, st>>>(vstride, sc, sh->yx, yfix, y);
        return CIH_OK;
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
        if ((rc = spmv(V + (int64_t)j * vstride, w))) break;
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


int ham_spmv(const cih_basis &b, const int64_t *rowptr, const int32_t *col, const float *val, int K, bool values_em,
             const double *x, double *y, cudaStream_t st)
{
    const int64_t dim = b.dim;
    if (dim == 0) return CIH_OK;
    if (K > kThreads) return fail(CIH_ERR_UNSUPPORTED, "spmv: at most 256 sets per call");
    if (dim > INT32_MAX) return fail(CIH_ERR_UNSUPPORTED, "spmv: dimension above 2^31");
    int64_t nnz = 0;
    if (K > 1 && !values_em) {
        cudaError_t e = cudaMemcpyAsync(&nnz, rowptr + dim, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "spmv: read nnz");
    }
    const int64_t n = dim * K;
    std::vector<void *> bufs;
    auto alloc = [&](void **p, size_t bytes) -> bool {
        if (cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), b.pool, st) != cudaSuccess) {
            (void)cudaGetLastError();
            return false;
        }
        bufs.push_back(*p);
        return true;
    };
    unsigned long long *yfix = nullptr;
    float2 *xs = nullptr, *xm = nullptr, *yrow = nullptr;
    double *partial = nullptr, *xpart = nullptr, *xn2 = nullptr, *sc = nullptr;
    float *vem = nullptr;
    bool ok = alloc((void **)&yfix, sizeof(unsigned long long) * (size_t)n) &&
              alloc((void **)&xs, sizeof(float2) * (size_t)n) && alloc((void **)&xm, sizeof(float2) * (size_t)n) &&
              alloc((void **)&yrow, sizeof(float2) * (size_t)n) &&
              alloc((void **)&partial, sizeof(double) * kDotBlocks) &&
              alloc((void **)&xpart, sizeof(double) * (size_t)K * kDotBlocks) &&
              alloc((void **)&xn2, sizeof(double) * K) && alloc((void **)&sc, sizeof(double) * 4);
    if (ok && K > 1 && !values_em) ok = alloc((void **)&vem, sizeof(float) * (size_t)nnz * K);
    int rc = ok ? CIH_OK : fail(CIH_ERR_NOMEM, "spmv: device memory");
    if (!rc) {
        if (K > 1 && !values_em) {
            count_launches(1);
            k_vals_em<<<grid_for(nnz * K), kThreads, 0, st>>>(K, nnz, val, vem);
        } else {
            vem = const_cast<float *>(val);
        }
        cudaMemsetAsync(yfix, 0, sizeof(unsigned long long) * (size_t)n, st);
        count_launches(6);
        k_upper_sumsq<<<kDotBlocks, kSumsqThreads, 0, st>>>(RowRange{0, dim, 0}, K, rowptr, vem, partial);
        k_dots<<<dim3(kDotBlocks, 1), kThreads, 0, st>>>(dim, K, 1, x, n, x, xpart);
        k_dots_finish<<<(K + 255) / 256, 256, 0, st>>>(K, kDotBlocks, xpart, xn2);
        k_mirror_scale<<<1, 32, 0, st>>>(kDotBlocks, partial, K, xn2, sc);
        k_split<<<grid_for(n), kThreads, 0, st>>>(n, x, sc, xs, xm);
        const int gr = (int)std::min<int64_t>((dim + 7) / 8, 152 * 32);
        launch_spmv(RowRange{0, dim, 0}, K, rowptr, col, vem, xs, xm, yrow, yfix, gr, st);
        k_sym_finish<<<grid_for(n), kThreads, 0, st>>>(n, sc, yrow, y, yfix);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "spmv kernels");
    }
    for (void *p : bufs) cudaFreeAsync(p, st);
    return rc;
}


int upper_sumsq(const cih_basis &b, const int64_t *rowptr, int64_t r0, int64_t r1, const float *val, int K,
                bool values_em, double *f2, cudaStream_t st)
{
    *f2 = 0.0;
    if (r1 <= r0) return CIH_OK;
    if (K > kThreads) return fail(CIH_ERR_UNSUPPORTED, "upper_sumsq: at most 256 sets per call");
    int64_t ends[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&ends[0], rowptr + r0, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ends[1], rowptr + r1, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "upper_sumsq: read nnz");
    const int64_t nnz = ends[1] - ends[0];
    float *vem = const_cast<float *>(val);
    double *partial = nullptr;
    if (cudaMallocFromPoolAsync((void **)&partial, sizeof(double) * kDotBlocks, b.pool, st) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(CIH_ERR_NOMEM, "upper_sumsq: device memory");
    }
    int rc = CIH_OK;
    if (K > 1 && !values_em) {
        if (cudaMallocFromPoolAsync((void **)&vem, std::max<size_t>(sizeof(float) * (size_t)nnz * K, 16), b.pool, st) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            cudaFreeAsync(partial, st);
            return fail(CIH_ERR_NOMEM, "upper_sumsq: device memory");
        }
        count_launches(1);
        k_vals_em<<<grid_for(nnz * K), kThreads, 0, st>>>(K, nnz, val, vem);
    }
    count_launches(1);
    k_upper_sumsq<<<kDotBlocks, kSumsqThreads, 0, st>>>(RowRange{r0, r1, ends[0]}, K, rowptr, vem, partial);
    std::vector<double> hp(kDotBlocks);
    e = cudaMemcpyAsync(hp.data(), partial, sizeof(double) * kDotBlocks, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "upper_sumsq");
    for (int k = 0; k < kDotBlocks && !rc; ++k) *f2 += hp[k];             // the order k_mirror_scale sums in
    cudaFreeAsync(partial, st);
    if (vem != val) cudaFreeAsync(vem, st);
    return rc;
}

}  // namespace cih

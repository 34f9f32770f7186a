// Device set-up of a basis: upload the host tables and build, per species,
// the neighbour lists the Hamiltonian kernels walk.
//
// Sec. 4.1 of the paper locates nonzeros either by testing every element of
// a dense block or, for sparse blocks, by iterating only over the quantum
// number combinations that can be nonzero.  Both appear here, one level
// down: the same-class forward list of a sub-determinant is found by testing
// every later member of its (2M, parity) class (XOR + popcount), and the
// one-move list by generating each single-orbital move and looking the result
// up in the sorted sub-determinant table.  Sec. 5.2's lesson (build index
// structures contiguously, one allocation each) applies to every list.
#include <algorithm>
#include <cstring>

#include "cih_internal.h"

namespace cih {
namespace {

struct SpeciesBuild {
    const uint64_t *bits;      // n_sd x W
    const int8_t *N;
    const int16_t *M2;
    const int32_t *cls_end;
    const int32_t *cls_lookup;  // (M2 + moff) * 2 + parity -> class id, -1 if none
    const int32_t *cls_begin;
    const int32_t *cls_endc;    // per class
    const int8_t *oN;           // per orbital
    const int16_t *om2;
    int32_t n_sd, n_orb, moff, mspan, Nsub_max;
};

template <int W>
__device__ __forceinline__ void load_bits(const uint64_t *base, int64_t i, uint64_t (&o)[W])
{
#pragma unroll
    for (int w = 0; w < W; ++w) o[w] = base[i * W + w];
}

template <int W>
__device__ __forceinline__ int xor_pop(const uint64_t (&a)[W], const uint64_t *b)
{
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += __popcll(a[w] ^ b[w]);
    return c;
}

// Same-class forward neighbours (1 or 2 orbitals moved, index > x): count or
// write, one warp per sub-det, lanes over the later class members.
template <int W, bool WRITE>
__global__ void k_forward(SpeciesBuild S, int64_t *cnt, const int64_t *off, int32_t *out)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < S.n_sd; x += nwarps) {
        uint64_t bx[W];
        load_bits<W>(S.bits, x, bx);
        int end = S.cls_end[x];
        int64_t pos = WRITE ? off[x] : 0;
        for (int y0 = (int)x + 1; y0 < end; y0 += 32) {
            int y = y0 + lane;
            bool hit = false;
            if (y < end) {
                int d = xor_pop<W>(bx, S.bits + (int64_t)y * W);
                hit = d <= 4;                          // d == 0 only for y == x
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            if (WRITE && hit) out[pos + __popc(m & ((1u << lane) - 1))] = y;
            pos += __popc(m);
        }
        if (!WRITE && lane == 0) cnt[x] = pos;
    }
}

// index of the sub-det with bits `yb`, quanta Ny and 2M My, or -1
template <int W>
__device__ int find_subdet(const SpeciesBuild &S, const uint64_t (&yb)[W], int Ny, int My)
{
    int key = My + S.moff;
    if (key < 0 || key >= S.mspan) return -1;
    int c = S.cls_lookup[key * 2 + (Ny & 1)];
    if (c < 0) return -1;
    int lo = S.cls_begin[c], hi = S.cls_endc[c];       // sorted by (N, bits)
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int Nm = S.N[mid];
        bool less;
        if (Nm != Ny) {
            less = Nm < Ny;
        } else {
            less = false;
            const uint64_t *mb = S.bits + (int64_t)mid * W;
#pragma unroll
            for (int w = W - 1; w >= 0; --w) {
                if (mb[w] != yb[w]) { less = mb[w] < yb[w]; break; }
            }
        }
        if (less) lo = mid + 1; else hi = mid;
    }
    if (lo >= S.cls_endc[c] || S.N[lo] != Ny) return -1;
    const uint64_t *mb = S.bits + (int64_t)lo * W;
#pragma unroll
    for (int w = 0; w < W; ++w)
        if (mb[w] != yb[w]) return -1;
    return lo;
}

// One-move neighbours: remove an occupied orbital r, add an empty orbital a;
// one warp per sub-det, lanes over a.  Written unsorted, sorted afterwards.
template <int W, bool WRITE>
__global__ void k_onemove(SpeciesBuild S, int64_t *cnt, const int64_t *off, int32_t *out)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < S.n_sd; x += nwarps) {
        uint64_t bx[W];
        load_bits<W>(S.bits, x, bx);
        int Nx = S.N[x];
        int Mx = S.M2[x];
        int64_t pos = WRITE ? off[x] : 0;
        for (int w = 0; w < W; ++w) {
            uint64_t occ = bx[w];
            while (occ) {
                int r = w * 64 + __ffsll((long long)occ) - 1;
                occ &= occ - 1;
                int Nr = S.oN[r], Mr = S.om2[r];
                for (int a0 = 0; a0 < S.n_orb; a0 += 32) {
                    int a = a0 + lane;
                    int found = -1;
                    if (a < S.n_orb && !((bx[a >> 6] >> (a & 63)) & 1)) {
                        int Ny = Nx - Nr + S.oN[a];
                        if (Ny <= S.Nsub_max) {
                            uint64_t yb[W];
#pragma unroll
                            for (int v = 0; v < W; ++v) yb[v] = bx[v];
                            yb[r >> 6] &= ~(1ull << (r & 63));
                            yb[a >> 6] |= 1ull << (a & 63);
                            found = find_subdet<W>(S, yb, Ny, Mx - Mr + S.om2[a]);
                        }
                    }
                    unsigned m = __ballot_sync(0xffffffffu, found >= 0);
                    if (WRITE && found >= 0) out[pos + __popc(m & ((1u << lane) - 1))] = found;
                    pos += __popc(m);
                }
            }
        }
        if (!WRITE && lane == 0) cnt[x] = pos;
    }
}

// Sort each list [off[x], off[x+1]) ascending: one block per list, bitonic
// sort in shared memory (lists are at most kSortTile long; checked on the host).
__global__ void k_sort_lists(const int64_t *off, int32_t *data, int64_t n)
{
    __shared__ int32_t s[kSortTile];
    for (int64_t x = blockIdx.x; x < n; x += gridDim.x) {
        int64_t b = off[x];
        int len = (int)(off[x + 1] - b);
        if (len <= 1) continue;
        int P = 1;
        while (P < len) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = i < len ? data[b + i] : INT32_MAX;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    int l = i ^ j;
                    if (l > i) {
                        bool up = (i & k) == 0;
                        int32_t a = s[i], c = s[l];
                        if ((a > c) == up) { s[i] = c; s[l] = a; }
                    }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < len; i += blockDim.x) data[b + i] = s[i];
        __syncthreads();
    }
}

template <class T>
int dev_alloc(cih_basis &b, T **p, size_t n)
{
    *p = nullptr;
    size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(CIH_ERR_NOMEM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    b.buffers.owned.push_back((void *)*p);
    return CIH_OK;
}

template <class T>
int upload(cih_basis &b, T **p, const std::vector<T> &h, cudaStream_t st)
{
    int rc = dev_alloc(b, p, h.size());
    if (rc) return rc;
    if (!h.empty()) {
        cudaError_t e = cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "upload");
    }
    return CIH_OK;
}

int grid_for(int64_t warps)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (warps + 7) / 8;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sms * 16));
}

template <int W>
int build_lists(cih_basis &b, int t, SpeciesBuild &S, cudaStream_t st)
{
    DevSpecies &D = b.dev.sp[t];
    int64_t n = S.n_sd;
    int64_t *cnt_fw, *cnt_n1, *scratch;
    int rc;
    if ((rc = dev_alloc(b, &cnt_fw, n + 1)) || (rc = dev_alloc(b, &cnt_n1, n + 1))) return rc;
    int64_t ns = scan_scratch_needed(n);
    if ((rc = dev_alloc(b, &scratch, ns))) return rc;
    int grid = grid_for(n);
    if (n > 0) {
        count_launches(2);
        k_forward<W, false><<<grid, 256, 0, st>>>(S, cnt_fw, nullptr, nullptr);
        k_onemove<W, false><<<grid, 256, 0, st>>>(S, cnt_n1, nullptr, nullptr);
    }
    if ((rc = exclusive_scan_i64(cnt_fw, n, scratch, ns, st))) return rc;
    if ((rc = exclusive_scan_i64(cnt_n1, n, scratch, ns, st))) return rc;
    int64_t tot[2];
    cudaMemcpyAsync(&tot[0], cnt_fw + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&tot[1], cnt_n1 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "neighbour count");
    int32_t *fw, *n1;
    if ((rc = dev_alloc(b, &fw, tot[0])) || (rc = dev_alloc(b, &n1, tot[1]))) return rc;
    if (n > 0) {
        count_launches(2);
        k_forward<W, true><<<grid, 256, 0, st>>>(S, nullptr, cnt_fw, fw);
        k_onemove<W, true><<<grid, 256, 0, st>>>(S, nullptr, cnt_n1, n1);
    }
    // the sort tile bounds the one-move list length: check it on the host
    std::vector<int64_t> hoff(n + 1);
    e = cudaMemcpyAsync(hoff.data(), cnt_n1, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "neighbour offsets");
    for (int64_t x = 0; x < n; ++x)
        if (hoff[x + 1] - hoff[x] > kSortTile) return fail(CIH_ERR_UNSUPPORTED, "one-move list longer than the sort tile");
    if (n > 0) count_launches(1);
    if (n > 0) k_sort_lists<<<(int)std::min<int64_t>(n, 65535), 256, 0, st>>>(cnt_n1, n1, n);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "neighbour kernels");
    D.fw_off = cnt_fw;
    D.fw = fw;
    D.n1_off = cnt_n1;
    D.n1 = n1;
    return CIH_OK;
}

}  // namespace

int upload_and_build_neighbours(cih_basis &b, cudaStream_t st)
{
    int rc;
    int W = b.W;
    for (int t = 0; t < 2; ++t) {
        const Species &s = b.s[t];
        // bit strings compacted to W words
        std::vector<uint64_t> bits((size_t)s.n_sd * W);
        for (int64_t i = 0; i < s.n_sd; ++i)
            for (int w = 0; w < W; ++w) bits[i * W + w] = s.bits[i * kMaxWords + w];
        std::vector<int8_t> N(s.N.begin(), s.N.end());
        std::vector<int16_t> M2(s.M2.begin(), s.M2.end());
        std::vector<int32_t> cls_end(s.n_sd);
        for (int64_t i = 0; i < s.n_sd; ++i) cls_end[i] = s.cls_end[s.cls[i]];
        int mabs = 0;
        for (int m : s.cls_M2) mabs = std::max(mabs, std::abs(m));
        int mspan = 2 * mabs + 1 + 64;          // room for moves that leave the table
        int moff = mabs + 32;
        std::vector<int32_t> lookup((size_t)mspan * 2, -1);
        for (size_t c = 0; c < s.cls_begin.size(); ++c)
            lookup[(size_t)(s.cls_M2[c] + moff) * 2 + s.cls_par[c]] = (int32_t)c;
        std::vector<int32_t> cb(s.cls_begin.begin(), s.cls_begin.end()), ce(s.cls_end.begin(), s.cls_end.end());
        std::vector<int8_t> oN(s.oN.begin(), s.oN.end());
        std::vector<int16_t> om2(s.om2.begin(), s.om2.end());

        uint64_t *d_bits; int8_t *d_N; int16_t *d_M2; int32_t *d_cls_end, *d_lookup, *d_cb, *d_ce;
        int8_t *d_oN; int16_t *d_om2;
        if ((rc = upload(b, &d_bits, bits, st)) || (rc = upload(b, &d_N, N, st)) ||
            (rc = upload(b, &d_M2, M2, st)) || (rc = upload(b, &d_cls_end, cls_end, st)) ||
            (rc = upload(b, &d_lookup, lookup, st)) || (rc = upload(b, &d_cb, cb, st)) ||
            (rc = upload(b, &d_ce, ce, st)) || (rc = upload(b, &d_oN, oN, st)) ||
            (rc = upload(b, &d_om2, om2, st)))
            return rc;
        DevSpecies &D = b.dev.sp[t];
        D.bits = d_bits;
        D.N = d_N;
        D.cls_end = d_cls_end;
        D.n_sd = (int32_t)s.n_sd;
        D.n_orb = s.n_orb;
        D.orb_base = t == 0 ? 0 : b.s[0].n_orb;

        SpeciesBuild S{d_bits, d_N, d_M2, d_cls_end, d_lookup, d_cb, d_ce, d_oN, d_om2,
                       (int32_t)s.n_sd, s.n_orb, moff, mspan, s.Nsub_max};
        if (W == 1) rc = build_lists<1>(b, t, S, st);
        else if (W == 2) rc = build_lists<2>(b, t, S, st);
        else rc = build_lists<4>(b, t, S, st);
        if (rc) return rc;
    }
    // basis-level tables
    int ntot = b.s[0].n_orb + b.s[1].n_orb;
    std::vector<int8_t> orbN(ntot);
    for (int a = 0; a < ntot; ++a) orbN[a] = (int8_t)(a < b.s[0].n_orb ? b.s[0].oN[a] : b.s[1].oN[a - b.s[0].n_orb]);
    int32_t *d_nb, *d_nc, *d_pid, *d_gsize;
    int64_t *d_rowbase, *d_goff;
    int8_t *d_orbN;
    if ((rc = upload(b, &d_nb, b.nb, st)) || (rc = upload(b, &d_nc, b.nc, st)) ||
        (rc = upload(b, &d_rowbase, b.rowbase, st)) || (rc = upload(b, &d_orbN, orbN, st)) ||
        (rc = upload(b, &d_pid, b.layout.pid, st)) || (rc = upload(b, &d_gsize, b.layout.gsize, st)) ||
        (rc = upload(b, &d_goff, b.layout.goff, st)))
        return rc;
    b.dev.nb = d_nb;
    b.dev.nc = d_nc;
    b.dev.rowbase = d_rowbase;
    b.dev.orbN = d_orbN;
    b.dev.pid = d_pid;
    b.dev.gsize = d_gsize;
    b.dev.goff = d_goff;
    b.dev.n_p = (int32_t)b.s[0].n_sd;
    b.dev.ntot = ntot;
    b.dev.dim = b.dim;
    b.dev.tbme_len = b.layout.total;
    b.scan_scratch_len = scan_scratch_needed(b.dim);
    if ((rc = dev_alloc(b, &b.scan_scratch, b.scan_scratch_len))) return rc;
    if ((rc = dev_alloc(b, &b.dev_status, 1))) return rc;
    cudaError_t e = cudaMemsetAsync(b.dev_status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "basis upload");
    return CIH_OK;
}

}  // namespace cih

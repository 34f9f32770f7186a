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

#include <functional>
#include <mutex>

#include "cih_internal.h"

namespace cih {
namespace {



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

template <int W>
__device__ __forceinline__ uint32_t hash_bits(const uint64_t *b)
{
    uint64_t h = 0x9E3779B97F4A7C15ull;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        h ^= b[w] + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
        h *= 0xBF58476D1CE4E5B9ull;
    }
    return (uint32_t)(h ^ (h >> 31));
}

// insert every sub-det index (all keys distinct: claim the first empty slot)
template <int W>
__global__ void k_hash_build(SpeciesBuild S, int32_t *table)
{
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < S.n_sd; x += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = hash_bits<W>(S.bits + x * W) & S.hash_mask;
        for (uint32_t probe = 0; probe <= S.hash_mask; ++probe) {
            if (atomicCAS(&table[h], -1, (int32_t)x) == -1) break;
            h = (h + 1) & S.hash_mask;
        }
    }
}

// index of the sub-det with bits `yb`, or -1 (hash lookup; at most capacity probes)
template <int W>
__device__ int find_subdet(const SpeciesBuild &S, const uint64_t (&yb)[W], int Ny, int My)
{
    (void)Ny;
    (void)My;
    uint32_t h = hash_bits<W>(yb) & S.hash_mask;
    for (uint32_t probe = 0; probe <= S.hash_mask; ++probe) {
        const int32_t x = S.hash[h];
        if (x < 0) return -1;
        const uint64_t *xb = S.bits + (int64_t)x * W;
        bool eq = true;
#pragma unroll
        for (int w = 0; w < W; ++w) eq &= xb[w] == yb[w];
        if (eq) return x;
        h = (h + 1) & S.hash_mask;
    }
    return -1;
}

// index of the sub-det with bits `yb`, quanta Ny and 2M My, or -1 (binary
// search inside its class; kept for reference)
template <int W>
__device__ int find_subdet_sorted(const SpeciesBuild &S, const uint64_t (&yb)[W], int Ny, int My)
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

template <int W>
__device__ __forceinline__ int low_bit(const uint64_t (&x)[W])
{
#pragma unroll
    for (int w = 0; w < W; ++w)
        if (x[w]) return w * 64 + __ffsll((long long)x[w]) - 1;
    return -1;
}

template <int W>
__device__ __forceinline__ int count_below(const uint64_t (&R)[W], int k)
{
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        int lo = w * 64;
        if (k >= lo + 64) c += __popcll(R[w]);
        else if (k > lo) c += __popcll(R[w] & ((1ull << (k - lo)) - 1));
    }
    return c;
}

// Packed one-move of each neutron list entry, bra x -> ket y:
//   b = orbital in x only, d = orbital in y only, R = common orbitals;
//   bits 0..7 r(d), 8..15 r(b), 16..22 2m_b + 64, 23 N_b & 1,
//   24 sign (-1)^(#R below b + #R below d).
template <int W>
__global__ void k_n1_info(SpeciesBuild S, const int64_t *off, const int32_t *list, const int32_t *rn,
                          uint32_t *info)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < S.n_sd; x += nwarps) {
        uint64_t bx[W];
        load_bits<W>(S.bits, x, bx);
        for (int64_t t = off[x] + lane; t < off[x + 1]; t += 32) {
            uint64_t by[W], R[W], dx[W], dy[W];
            load_bits<W>(S.bits, list[t], by);
#pragma unroll
            for (int w = 0; w < W; ++w) { R[w] = bx[w] & by[w]; dx[w] = bx[w] & ~by[w]; dy[w] = by[w] & ~bx[w]; }
            int b = low_bit<W>(dx), d = low_bit<W>(dy);
            int sg = (count_below<W>(R, b) + count_below<W>(R, d)) & 1;
            info[t] = (uint32_t)rn[d] | ((uint32_t)rn[b] << 8) | ((uint32_t)(S.om2[b] + 64) << 16) |
                      ((uint32_t)(S.oN[b] & 1) << 23) | ((uint32_t)sg << 24);
        }
    }
}

// Table index (<< 1) and sign bit of the two-move of each forward entry,
// bra x -> ket y; one-moves are stored as ~(b | d << 8 | sign << 16) with b
// in x only, d in y only.  Orbitals are offset by `base` into the
// combined index of the pair table.
template <int W>
__global__ void k_fw_tb(SpeciesBuild S, int base, const int64_t *off, const int32_t *list, const int32_t *pid,
                        const int32_t *gsize, const int64_t *goff, int ntot, int32_t *tb, int *status)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < S.n_sd; x += nwarps) {
        uint64_t bx[W];
        load_bits<W>(S.bits, x, bx);
        for (int64_t t = off[x] + lane; t < off[x + 1]; t += 32) {
            uint64_t by[W], R[W], dx[W], dy[W];
            load_bits<W>(S.bits, list[t], by);
            int pc = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                R[w] = bx[w] & by[w]; dx[w] = bx[w] & ~by[w]; dy[w] = by[w] & ~bx[w];
                pc += __popcll(dx[w]);
            }
            if (pc != 2) {                                  // one-move: ~(b | d << 8 | sign << 16)
                const int b1 = low_bit<W>(dx), d1 = low_bit<W>(dy);
                const int s1 = (count_below<W>(R, b1) + count_below<W>(R, d1)) & 1;
                tb[t] = ~(int32_t)(b1 | (d1 << 8) | (s1 << 16));
                continue;
            }
            int a1 = low_bit<W>(dx); dx[a1 >> 6] &= ~(1ull << (a1 & 63));
            int a2 = low_bit<W>(dx);
            int c1 = low_bit<W>(dy); dy[c1 >> 6] &= ~(1ull << (c1 & 63));
            int c2 = low_bit<W>(dy);
            int sg = (count_below<W>(R, a1) + count_below<W>(R, a2) + count_below<W>(R, c1) + count_below<W>(R, c2)) & 1;
            int32_t e1 = pid[(base + a1) * ntot + base + a2], e2 = pid[(base + c1) * ntot + base + c2];
            if (e1 < 0 || e2 < 0 || ((e1 ^ e2) & (0xFFF << 16))) { atomicOr(status, 4); tb[t] = -1; continue; }
            int g = (e1 >> 16) & 0xFFF;
            int64_t u = e1 & 0xFFFF, v = e2 & 0xFFFF;
            if (u > v) { int64_t q = u; u = v; v = q; }
            int64_t n = gsize[g];
            int64_t idx = goff[g] + u * n - u * (u - 1) / 2 + (v - u);
            tb[t] = (int32_t)((idx << 1) | sg);
        }
    }
}

// first one-move entry of each sub-det beyond its own class, and the size of
// its candidate list (forward same-class entries + later-class one-moves)
__global__ void k_later(int64_t n, const int32_t *cls_end, const int64_t *fw_off, const int64_t *n1_off,
                        const int32_t *n1, int64_t *later, int *max_cand)
{
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = n1_off[x], hi = n1_off[x + 1];
        int key = cls_end[x];
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (n1[mid] < key) lo = mid + 1; else hi = mid;
        }
        later[x] = lo;
        int64_t c = (fw_off[x + 1] - fw_off[x]) + (n1_off[x + 1] - lo);
        atomicMax(max_cand, (int)min(c, (int64_t)INT32_MAX));
    }
}

// Candidate table of proton sub-det p (bra p -> ket q); see DevBasis.
// The directory indices locate q's neutron range in the one-move list of any
// row neutron n of p: the range is the prefix N <= L_q of the class
// (2M - 2M_q, parity of Nlim - N_q), which relative to n's class is
// 2M_p - 2M_q.
template <int W>
__global__ void k_cand(SpeciesBuild S, DevBasis B, const int8_t *Nq, const int16_t *M2q, int Nlim, int64_t *cand_off,
                       int4 *cand, uint8_t *cself)
{
    const DevSpecies &SP = B.sp[0];
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int G = B.pn_G, span = B.pn_m2span, NL = B.NL, DM = B.DM;
    for (int64_t p = warp; p < S.n_sd; p += nwarps) {
        uint64_t pb[W];
        load_bits<W>(S.bits, p, pb);
        const int64_t f0 = SP.fw_off[p], nf = SP.fw_off[p + 1] - f0;
        const int64_t l0 = SP.n1_later[p];
        const int64_t C = nf + (SP.n1_off[p + 1] - l0);
        const int64_t base = cand_off[p];
        const int par_p = (Nlim - Nq[p]) & 1;
        for (int64_t k = lane; k < C; k += 32) {
            const int q = k < nf ? SP.fw[f0 + k] : SP.n1[l0 + (k - nf)];
            uint64_t qb[W], R[W], dx[W], dy[W];
            load_bits<W>(S.bits, q, qb);
            int pc = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                R[w] = pb[w] & qb[w]; dx[w] = pb[w] & ~qb[w]; dy[w] = qb[w] & ~pb[w];
                pc += __popcll(dx[w]);
            }
            const int Lq = Nlim - Nq[q];                       // largest N of a partner of q
            const int par_q = Lq & 1;
            const int dM = M2q[p] - M2q[q];
            const int rc = ((dM + DM) >> 1) * 2 + par_q;
            const int Lc = min(Lq, NL - 1);
            int st = rc * NL, en = 1 + rc * NL + Lc;
            if (dM > DM || dM < -DM || Lc < 0) st = en = 0;  // no neutron one-move reaches q's range
            const bool same = M2q[p] == M2q[q] && par_p == par_q;    // q's range is in n's class
            int4 r;
            r.x = (int32_t)(B.rowbase[q] - B.nb[q]);
            r.y = st | (en << 16);
            uint8_t sl = same ? (uint8_t)(1 + Lq) : 0;
            if (pc == 1) {
                const int a = low_bit<W>(dx), c = low_bit<W>(dy);
                const int sg = (count_below<W>(R, a) + count_below<W>(R, c)) & 1;
                const int Ka = (S.om2[a] + span) & 0xFF;       // >= 0 by the choice of span
                r.z = (int32_t)((uint32_t)(a * G + Ka) | ((uint32_t)(c * G + Ka) << 16));
                r.w = (int32_t)((uint32_t)Ka | ((uint32_t)(S.oN[a] & 1) << 8) | ((uint32_t)sg << 9) |
                                ((uint32_t)a << 16) | ((uint32_t)c << 24));
            } else {
                r.z = B.fw_tb[0][f0 + k];
                r.w = 0;
                sl |= 0x80;
            }
            cand[base + k] = r;
            cself[base + k] = sl;
        }
    }
}

// occupied orbitals of each sub-det, ascending; and for the neutron lists the
// number of one-move entries below the sub-det itself
template <int W>
__global__ void k_occ(SpeciesBuild S, int Z, const int64_t *n1_off, const int32_t *n1, uint8_t *occ, int16_t *self_rel)
{
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < S.n_sd; x += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        for (int w = 0; w < W; ++w) {
            uint64_t m = S.bits[x * W + w];
            while (m) {
                occ[x * Z + k++] = (uint8_t)(w * 64 + __ffsll((long long)m) - 1);
                m &= m - 1;
            }
        }
        if (self_rel) {
            int64_t lo = n1_off[x], hi = n1_off[x + 1];
            const int64_t a0 = lo;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (n1[mid] < x) lo = mid + 1; else hi = mid;
            }
            self_rel[x] = (int16_t)(lo - a0);
        }
    }
}

// Pack each neutron one-move entry with its move info, and build the bucket
// directory of each list (see DevBasis).
__global__ void k_n1_pack(int64_t n, const int64_t *off, const int32_t *list, const uint32_t *info, int2 *packed)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < off[n]; t += (int64_t)gridDim.x * blockDim.x)
        packed[t] = make_int2(list[t], (int)info[t]);
}

__global__ void k_dir(SpeciesBuild S, const int64_t *off, const int32_t *list, int NL, int DM, int dir_len,
                      int16_t *dir)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < S.n_sd; x += nwarps) {
        const int64_t a0 = off[x], a1 = off[x + 1];
        const int M0 = S.M2[x];
        int16_t *d = dir + x * (int64_t)dir_len;
        if (lane == 0) d[0] = 0;
        for (int b = lane; b < dir_len - 1; b += 32) {
            // entries with bucket key <= b: keys are non-decreasing along the sorted list
            int64_t lo = a0, hi = a1;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int y = list[mid];
                const int key = (((int)S.M2[y] - M0 + DM) >> 1) * 2 * NL + (S.N[y] & 1) * NL + S.N[y];
                if (key <= b) lo = mid + 1; else hi = mid;
            }
            d[1 + b] = (int16_t)(lo - a0);
        }
    }
}

__global__ void k_cand_count(int64_t n, const int64_t *fw_off, const int64_t *n1_off, const int64_t *later,
                             int64_t *cnt)
{
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
        cnt[x] = (fw_off[x + 1] - fw_off[x]) + (n1_off[x + 1] - later[x]);
}

__global__ void k_row_p(int64_t np, const int64_t *rowbase, int32_t *row_p)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < np; p += nwarps)
        for (int64_t r = rowbase[p] + lane; r < rowbase[p + 1]; r += 32) row_p[r] = (int32_t)p;
}

// Single-pass forward lists: sub-det x at rank r of a class [cb, ce) of size
// m has room for m - r - 1 entries at stage offset
//   class_stage[c] + r (m - 1) - r (r - 1) / 2,
// written in ascending order; cnt[x] gets the count.
template <int W>
__global__ void k_forward_staged(SpeciesBuild S, const int32_t *cls_of, const int64_t *class_stage, int64_t *cnt,
                                 int32_t *stage)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < S.n_sd; x += nwarps) {
        uint64_t bx[W];
        load_bits<W>(S.bits, x, bx);
        const int c = cls_of[x];
        const int64_t cb = S.cls_begin[c], m = S.cls_endc[c] - cb, r = x - cb;
        int32_t *out = stage + class_stage[c] + r * (m - 1) - r * (r - 1) / 2;
        const int end = S.cls_end[x];
        int64_t pos = 0;
        for (int y0 = (int)x + 1; y0 < end; y0 += 32) {
            const int y = y0 + lane;
            bool hit = false;
            if (y < end) {                               // word-major copy: the warp's reads coalesce
                int d = 0;
#pragma unroll
                for (int w = 0; w < W; ++w) d += __popcll(bx[w] ^ S.bitsT[(int64_t)w * S.n_sd + y]);
                hit = d <= 4;
            }
            const unsigned msk = __ballot_sync(0xffffffffu, hit);
            if (hit) out[pos + __popc(msk & ((1u << lane) - 1))] = y;
            pos += __popc(msk);
        }
        if (lane == 0) cnt[x] = pos;
    }
}

// bitsT[w * n + x] = bits[x * W + w]
__global__ void k_bits_T(int64_t n, int W, const uint64_t *bits, uint64_t *bitsT)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * W; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = t / W;
        const int w = (int)(t - x * W);
        bitsT[(int64_t)w * n + x] = bits[t];
    }
}

__global__ void k_forward_compact(SpeciesBuild S, const int32_t *cls_of, const int64_t *class_stage,
                                  const int64_t *off, const int32_t *stage, int32_t *out)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < S.n_sd; x += nwarps) {
        const int c = cls_of[x];
        const int64_t cb = S.cls_begin[c], m = S.cls_endc[c] - cb, r = x - cb;
        const int32_t *in = stage + class_stage[c] + r * (m - 1) - r * (r - 1) / 2;
        const int64_t o = off[x], len = off[x + 1] - o;
        for (int64_t i = lane; i < len; i += 32) out[o + i] = in[i];
    }
}

// Single-pass one-move lists: each sub-det writes its moves (unsorted) into
// a slot of `cap` entries; cnt[x] gets the count.
template <int W>
__global__ void k_onemove_staged(SpeciesBuild S, int cap, int64_t *cnt, int32_t *stage)
{
    int lane = threadIdx.x & 31;
    int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = warp; x < S.n_sd; x += nwarps) {
        uint64_t bx[W];
        load_bits<W>(S.bits, x, bx);
        const int Nx = S.N[x];
        int32_t *out = stage + x * (int64_t)cap;
        int pos = 0;
        for (int w = 0; w < W; ++w) {
            uint64_t occ = bx[w];
            while (occ) {
                const int r = w * 64 + __ffsll((long long)occ) - 1;
                occ &= occ - 1;
                const int Nr = S.oN[r];
                // targets a with Nx - Nr + N_a <= Nsub_max: a prefix of the shell-ordered orbitals
                const int lim = S.Nsub_max - Nx + Nr;
                const int aend = lim < 0 ? 0 : lim >= S.maxN ? S.n_orb : S.orb_upto[lim];
                for (int a0 = 0; a0 < aend; a0 += 32) {
                    const int a = a0 + lane;
                    int found = -1;
                    if (a < aend && !((bx[a >> 6] >> (a & 63)) & 1) && Nx - Nr + S.oN[a] <= S.Nsub_max) {
                        uint64_t yb[W];
#pragma unroll
                        for (int v = 0; v < W; ++v) yb[v] = bx[v];
                        yb[r >> 6] &= ~(1ull << (r & 63));
                        yb[a >> 6] |= 1ull << (a & 63);
                        found = find_subdet<W>(S, yb, 0, 0);
                    }
                    const unsigned msk = __ballot_sync(0xffffffffu, found >= 0);
                    if (found >= 0) out[pos + __popc(msk & ((1u << lane) - 1))] = found;
                    pos += __popc(msk);
                }
            }
        }
        if (lane == 0) cnt[x] = pos;
    }
}

// one block per list: bitonic sort of the staged moves in shared memory,
// written compact at off[x]
__global__ void k_onemove_compact_sort(int64_t n, int cap, const int64_t *off, const int32_t *stage, int32_t *out)
{
    __shared__ int32_t sh[kSortTile];
    for (int64_t x = blockIdx.x; x < n; x += gridDim.x) {
        const int64_t o = off[x];
        const int len = (int)(off[x + 1] - o);
        const int32_t *in = stage + x * (int64_t)cap;
        if (len <= 32) {                          // small lists: one warp, insertion by rank
            if (threadIdx.x < 32) {
                const int32_t v = threadIdx.x < len ? in[threadIdx.x] : INT32_MAX;
                int rank = 0;
                for (int j = 0; j < len; ++j) {
                    const int32_t u = __shfl_sync(0xffffffffu, v, j);
                    rank += (u < v);
                }
                if ((int)threadIdx.x < len) out[o + rank] = v;
            }
            continue;
        }
        int P = 1;
        while (P < len) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) sh[i] = i < len ? in[i] : INT32_MAX;
        __syncthreads();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < P; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l > i) {
                        const bool up = (i & k) == 0;
                        const int32_t a = sh[i], c = sh[l];
                        if ((a > c) == up) { sh[i] = c; sh[l] = a; }
                    }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < len; i += blockDim.x) out[o + i] = sh[i];
        __syncthreads();
    }
}


// Count lists (see DevBasis): one warp per proton sub-det accumulates the
// directory coefficients of its one-move candidates (segment end +1, start
// -1) and the histogram of its candidates' 1 + L_q in shared memory; pass 0
// writes the number of non-zero coefficients, pass 1 the list (ascending
// directory position) and the suffix counts #{c : 1 + L_q(c) > N}.
constexpr int kClistDirCap = 4096;
template <int PASS>
__global__ void k_clists(int64_t np, const int64_t *cand_off, const int4 *cand, const uint8_t *cself, int dir_len,
                         int NL, int64_t *clen, const int64_t *clist_off, int2 *clist, uint16_t *cself_sfx)
{
    extern __shared__ int cl_sh[];                 // per warp: int[dir_len] coefficients, int[64] histogram
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int *coef = cl_sh + wid * (dir_len + 64);
    int *hist = coef + dir_len;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < np; p += nw) {
        for (int i = lane; i < dir_len; i += 32) coef[i] = 0;
        for (int i = lane; i < 64; i += 32) hist[i] = 0;
        __syncwarp();
        for (int64_t c = cand_off[p] + lane; c < cand_off[p + 1]; c += 32) {
            const uint8_t sl = cself[c];
            atomicAdd(&hist[min(sl & 0x7F, 63)], 1);              // > N for every N < NL either way
            if (!(sl >> 7)) {                                  // one-move: a neutron segment
                const unsigned y = (unsigned)cand[c].y;
                atomicAdd(&coef[y >> 16], 1);
                atomicAdd(&coef[y & 0xFFFF], -1);
            }
        }
        __syncwarp();
        int64_t out = PASS == 1 ? clist_off[p] : 0;
        int n = 0;
        for (int i0 = 0; i0 < dir_len; i0 += 32) {
            const int i = i0 + lane;
            const int v = i < dir_len ? coef[i] : 0;
            const unsigned m = __ballot_sync(0xffffffffu, v != 0);
            if (PASS == 1 && v != 0) clist[out + n + __popc(m & ((1u << lane) - 1))] = make_int2(i, v);
            n += __popc(m);
        }
        if (PASS == 0 && lane == 0) clen[p] = n;
        if (PASS == 1)
            for (int N = lane; N < NL; N += 32) {              // candidates with 1 + L_q > N
                int s = 0;
                for (int v = N + 1; v < 64; ++v) s += hist[v];
                cself_sfx[p * NL + N] = (uint16_t)s;
            }
        __syncwarp();
    }
}

template <class T>
int dev_alloc(cih_basis &b, T **p, size_t n)
{
    *p = nullptr;
    size_t bytes = (std::max<size_t>(n, 1) * sizeof(T) + 255) / 256 * 256;
    cudaError_t e = cudaMallocFromPoolAsync((void **)p, bytes, b.pool, b.stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
        return fail(CIH_ERR_NOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
    b.buffers.owned.push_back((void *)*p);
    return CIH_OK;
}

// return a buffer to the pool once the stream has passed its last use
template <class T>
void dev_free(cih_basis &b, T *p)
{
    if (!p) return;
    auto &v = b.buffers.owned;
    for (size_t i = 0; i < v.size(); ++i)
        if (v[i] == (void *)p) { v.erase(v.begin() + i); break; }
    cudaFreeAsync((void *)p, b.stream);
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

// Neighbour lists of one species, in three phases so that both species'
// kernels queue back to back and the host work in between overlaps them:
//   1. staged forward and one-move passes, their counts scanned, list totals
//      copied to pinned host memory;
//   2. (after one synchronisation) exact-size lists: compaction and sort,
//      later-entry offsets;
//   3. (once the table layout is on the device) two-move table indices and
//      the packed neutron move information.
struct Lists {
    int64_t n = 0, ns = 0;
    int64_t *cnt_fw = nullptr, *cnt_n1 = nullptr, *scratch = nullptr, *d_class_stage = nullptr;
    int32_t *d_cls_of = nullptr, *fw_st = nullptr, *n1_st = nullptr, *fw = nullptr, *n1 = nullptr;
    int64_t *later = nullptr;
    int *dmax = nullptr;
    int cap1 = 1, grid = 1;
    int64_t *tot = nullptr;                   // pinned: forward and one-move totals
    int32_t *rn = nullptr;                    // neutron species: pn split row of each orbital (device)
};

template <int W>
int lists_phase1(cih_basis &b, int t, SpeciesBuild &S, Lists &L, cudaStream_t st)
{
    const Species &hs = b.s[t];
    const int64_t n = L.n = S.n_sd;
    int rc;
    if ((rc = dev_alloc(b, &L.cnt_fw, n + 1)) || (rc = dev_alloc(b, &L.cnt_n1, n + 1))) return rc;
    L.ns = scan_scratch_needed(n);
    if ((rc = dev_alloc(b, &L.scratch, L.ns))) return rc;
    L.grid = grid_for(n);
    // staging: forward lists by class triangle, one-move lists by fixed slots
    std::vector<int32_t> cls_of(std::max<int64_t>(n, 1));
    std::vector<int64_t> class_stage(std::max<size_t>(hs.cls_begin.size(), 1));
    int64_t fw_stage = 0;
    for (size_t c = 0; c < hs.cls_begin.size(); ++c) {
        const int64_t m = hs.cls_end[c] - hs.cls_begin[c];
        class_stage[c] = fw_stage;
        fw_stage += m * (m - 1) / 2;
        for (int64_t x = hs.cls_begin[c]; x < hs.cls_end[c]; ++x) cls_of[x] = (int32_t)c;
    }
    L.cap1 = std::max(1, hs.Z * std::max(0, hs.n_orb - hs.Z));
    if (L.cap1 > kSortTile) return fail(CIH_ERR_UNSUPPORTED, "one-move lists longer than the sort tile");
    if ((rc = upload(b, &L.d_cls_of, cls_of, st)) || (rc = upload(b, &L.d_class_stage, class_stage, st)) ||
        (rc = dev_alloc(b, &L.fw_st, fw_stage)) || (rc = dev_alloc(b, &L.n1_st, (size_t)n * L.cap1)))
        return rc;
    if (n > 0) {
        count_launches(2);
        k_forward_staged<W><<<L.grid, 256, 0, st>>>(S, L.d_cls_of, L.d_class_stage, L.cnt_fw, L.fw_st);
        k_onemove_staged<W><<<L.grid, 256, 0, st>>>(S, L.cap1, L.cnt_n1, L.n1_st);
    }
    if ((rc = exclusive_scan_i64(L.cnt_fw, n, L.scratch, L.ns, st))) return rc;
    if ((rc = exclusive_scan_i64(L.cnt_n1, n, L.scratch, L.ns, st))) return rc;
    cudaMemcpyAsync(&L.tot[0], L.cnt_fw + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&L.tot[1], L.cnt_n1 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    return CIH_OK;
}

int lists_phase2(cih_basis &b, int t, SpeciesBuild &S, Lists &L, cudaStream_t st)
{
    const int64_t n = L.n;
    int rc;
    if ((rc = dev_alloc(b, &L.fw, L.tot[0])) || (rc = dev_alloc(b, &L.n1, L.tot[1]))) return rc;
    if (n > 0) {
        count_launches(2);
        k_forward_compact<<<L.grid, 256, 0, st>>>(S, L.d_cls_of, L.d_class_stage, L.cnt_fw, L.fw_st, L.fw);
        k_onemove_compact_sort<<<(int)std::min<int64_t>(n, 65535), 256, 0, st>>>(n, L.cap1, L.cnt_n1, L.n1_st, L.n1);
    }
    dev_free(b, L.fw_st);
    dev_free(b, L.n1_st);
    L.fw_st = L.n1_st = nullptr;
    if ((rc = dev_alloc(b, &L.later, n)) || (rc = dev_alloc(b, &L.dmax, 1))) return rc;
    cudaMemsetAsync(L.dmax, 0, sizeof(int), st);
    if (n > 0) {
        count_launches(1);
        k_later<<<L.grid, 256, 0, st>>>(n, S.cls_end, L.cnt_fw, L.cnt_n1, L.n1, L.later, L.dmax);
    }
    DevSpecies &D = b.dev.sp[t];
    D.fw_off = L.cnt_fw;
    D.fw = L.fw;
    D.n1_off = L.cnt_n1;
    D.n1 = L.n1;
    D.n1_later = L.later;
    return CIH_OK;
}

template <int W>
int lists_phase3(cih_basis &b, int t, SpeciesBuild &S, Lists &L, cudaStream_t st)
{
    const int64_t n = L.n;
    int rc;
    int32_t *tb;
    if ((rc = dev_alloc(b, &tb, L.tot[0]))) return rc;
    if (n > 0) {
        count_launches(1);
        k_fw_tb<W><<<L.grid, 256, 0, st>>>(S, t == 0 ? 0 : b.s[0].n_orb, L.cnt_fw, L.fw, b.dev.pid, b.dev.gsize,
                                           b.dev.goff, b.dev.ntot, tb, b.dev_status);
    }
    if (t == 1) {
        uint32_t *info;
        if ((rc = dev_alloc(b, &info, L.tot[1]))) return rc;
        if (n > 0) {
            count_launches(1);
            k_n1_info<W><<<L.grid, 256, 0, st>>>(S, L.cnt_n1, L.n1, L.rn, info);
        }
        b.dev.n1_info = info;
    }
    if (t == 0) cudaMemcpyAsync(&L.tot[2], L.dmax, sizeof(int), cudaMemcpyDeviceToHost, st);
    b.dev.fw_tb[t] = tb;
    return CIH_OK;
}

// species t: host arrays (built for both species side by side), then their
// upload and the one-move hash table
struct SpeciesHost {
    std::vector<uint64_t> bits;
    std::vector<int8_t> N, oN;
    std::vector<int16_t> M2, om2;
    std::vector<int32_t> cls_end, lookup, cb, ce;
    int moff = 0, mspan = 0;
};

void species_prep(const cih_basis &b, int t, SpeciesHost &H)
{
    const int W = b.W;
    const Species &s = b.s[t];
    H.bits.resize((size_t)s.n_sd * W);               // bit strings compacted to W words
    for (int64_t i = 0; i < s.n_sd; ++i)
        for (int w = 0; w < W; ++w) H.bits[i * W + w] = s.bits[i * kMaxWords + w];
    H.N.assign(s.N.begin(), s.N.end());
    H.M2.assign(s.M2.begin(), s.M2.end());
    H.cls_end.resize(s.n_sd);
    for (int64_t i = 0; i < s.n_sd; ++i) H.cls_end[i] = s.cls_end[s.cls[i]];
    int mabs = 0;
    for (int m : s.cls_M2) mabs = std::max(mabs, std::abs(m));
    H.mspan = 2 * mabs + 1 + 64;                     // room for moves that leave the table
    H.moff = mabs + 32;
    H.lookup.assign((size_t)H.mspan * 2, -1);
    for (size_t c = 0; c < s.cls_begin.size(); ++c)
        H.lookup[(size_t)(s.cls_M2[c] + H.moff) * 2 + s.cls_par[c]] = (int32_t)c;
    H.cb.assign(s.cls_begin.begin(), s.cls_begin.end());
    H.ce.assign(s.cls_end.begin(), s.cls_end.end());
    H.oN.assign(s.oN.begin(), s.oN.end());
    H.om2.assign(s.om2.begin(), s.om2.end());
}

int species_upload(cih_basis &b, int t, const SpeciesHost &H, cudaStream_t st)
{
    const int W = b.W;
    const Species &s = b.s[t];
    int rc;
    uint64_t *d_bits; int8_t *d_N; int16_t *d_M2; int32_t *d_cls_end, *d_lookup, *d_cb, *d_ce;
    int8_t *d_oN; int16_t *d_om2;
    if ((rc = upload(b, &d_bits, H.bits, st)) || (rc = upload(b, &d_N, H.N, st)) ||
        (rc = upload(b, &d_M2, H.M2, st)) || (rc = upload(b, &d_cls_end, H.cls_end, st)) ||
        (rc = upload(b, &d_lookup, H.lookup, st)) || (rc = upload(b, &d_cb, H.cb, st)) ||
        (rc = upload(b, &d_ce, H.ce, st)) || (rc = upload(b, &d_oN, H.oN, st)) ||
        (rc = upload(b, &d_om2, H.om2, st)))
        return rc;
    DevSpecies &D = b.dev.sp[t];
    D.bits = d_bits;
    D.N = d_N;
    D.cls_end = d_cls_end;
    D.n_sd = (int32_t)s.n_sd;
    D.n_orb = s.n_orb;
    D.orb_base = t == 0 ? 0 : b.s[0].n_orb;

    SpeciesBuild S{d_bits, d_N, d_M2, d_cls_end, d_lookup, d_cb, d_ce, d_oN, d_om2,
                   (int32_t)s.n_sd, s.n_orb, H.moff, H.mspan, s.Nsub_max, nullptr, 0};
    uint32_t cap = 64;
    while (cap < 2 * (uint64_t)s.n_sd) cap <<= 1;
    int32_t *table;
    if ((rc = dev_alloc(b, &table, cap))) return rc;
    if (cudaMemsetAsync(table, 0xFF, sizeof(int32_t) * cap, st) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "hash table");
    S.hash = table;
    S.hash_mask = cap - 1;
    uint64_t *bitsT;
    if ((rc = dev_alloc(b, &bitsT, std::max<size_t>((size_t)s.n_sd * W, 1)))) return rc;
    if (s.n_sd > 0) {
        count_launches(1);
        k_bits_T<<<grid_for(((int64_t)s.n_sd * W + 31) / 32), 256, 0, st>>>(s.n_sd, W, d_bits, bitsT);
    }
    S.bitsT = bitsT;
    int maxN = 0;
    for (int a = 0; a < s.n_orb; ++a) maxN = std::max(maxN, s.oN[a]);
    std::vector<int32_t> upto(maxN + 1, 0);
    for (int a = 0; a < s.n_orb; ++a) upto[s.oN[a]] += 1;
    for (int k = 1; k <= maxN; ++k) upto[k] += upto[k - 1];
    for (int a = 1; a < s.n_orb; ++a)
        if (s.oN[a] < s.oN[a - 1]) return fail(CIH_ERR_UNSUPPORTED, "orbitals not ordered by shell");
    int32_t *d_upto;
    if ((rc = upload(b, &d_upto, upto, st))) return rc;
    S.orb_upto = d_upto;
    S.maxN = maxN;
    const int hg = (int)std::min<int64_t>((s.n_sd + 255) / 256 + 1, 65535);
    count_launches(1);
    if (W == 1) k_hash_build<1><<<hg, 256, 0, st>>>(S, table);
    else if (W == 2) k_hash_build<2><<<hg, 256, 0, st>>>(S, table);
    else k_hash_build<4><<<hg, 256, 0, st>>>(S, table);
    b.sbuild[t] = S;
    return CIH_OK;
}

// tables that need the partner ranges, the table layout and the pn split
int basis_tables_upload(cih_basis &b, cudaStream_t st)
{
    int rc;
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
    b.dev.ngroups = (int32_t)b.layout.gsize.size();
    b.dev.n_p = (int32_t)b.s[0].n_sd;
    b.dev.ntot = ntot;
    b.dev.dim = b.dim;
    b.dev.tbme_len = b.layout.total;
    std::vector<int8_t> m2p(std::max(b.s[0].n_orb, 1), 0), Np(std::max(b.s[0].n_orb, 1), 0);
    for (int a = 0; a < b.s[0].n_orb; ++a) { m2p[a] = (int8_t)b.s[0].om2[a]; Np[a] = (int8_t)b.s[0].oN[a]; }
    int16_t *d_S; int32_t *d_gs, *d_go; int8_t *d_m2p, *d_Np;
    if ((rc = upload(b, &d_S, b.pn.S, st)) || (rc = upload(b, &d_gs, b.pn.gsize, st)) ||
        (rc = upload(b, &d_go, b.pn.goff, st)) || (rc = upload(b, &d_m2p, m2p, st)) ||
        (rc = upload(b, &d_Np, Np, st)))
        return rc;
    b.dev.pn_S = d_S; b.dev.pn_gsize = d_gs; b.dev.pn_goff = d_go; b.dev.m2p = d_m2p; b.dev.Np = d_Np;
    b.dev.pn_G = b.pn.G;
    b.dev.pn_m2span = b.pn.m2span;
    int16_t *d_obg, *d_obl; int32_t *d_obs, *d_obo;
    if ((rc = upload(b, &d_obg, b.onebody.grp, st)) || (rc = upload(b, &d_obl, b.onebody.loc, st)) ||
        (rc = upload(b, &d_obs, b.onebody.gsize, st)) || (rc = upload(b, &d_obo, b.onebody.goff, st)))
        return rc;
    b.dev.ob_grp = d_obg; b.dev.ob_loc = d_obl; b.dev.ob_gsize = d_obs; b.dev.ob_goff = d_obo;
    return CIH_OK;
}

// Page-locked 8-word slots for the totals read back during set-up, kept for the
// next basis (allocating and freeing pinned memory costs more than the set-up's
// own synchronisations).
std::mutex g_slot_mu;
std::vector<int64_t *> g_slots;

struct PinnedTotals {
    int64_t *p = nullptr;
    cudaStream_t st = nullptr;                // copies into the slot are queued here
    cudaError_t get()
    {
        {
            std::lock_guard<std::mutex> lock(g_slot_mu);
            if (!g_slots.empty()) {
                p = g_slots.back();
                g_slots.pop_back();
                return cudaSuccess;
            }
        }
        cudaError_t e = cudaHostAlloc((void **)&p, 8 * sizeof(int64_t), cudaHostAllocPortable);   // any device
        if (e != cudaSuccess) p = nullptr;
        return e;
    }
    ~PinnedTotals()
    {
        if (!p) return;
        cudaStreamSynchronize(st);            // no copy still in flight into a returned slot
        std::lock_guard<std::mutex> lock(g_slot_mu);
        g_slots.push_back(p);
    }
};

// A second stream for the neutron species' list passes, which depend on the
// proton species' only through the candidate table.  The destructor waits for
// it, so that no early return leaves its kernels running on buffers the basis
// then frees.
struct SideStream {
    cudaStream_t s = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    cudaError_t create()
    {
        cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e != cudaSuccess) { s = nullptr; return e; }
        for (auto &x : ev)
            if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess) { x = nullptr; return e; }
        return cudaSuccess;
    }
    ~SideStream()
    {
        if (s) cudaStreamSynchronize(s);
        for (auto x : ev)
            if (x) cudaEventDestroy(x);
        if (s) cudaStreamDestroy(s);
    }
};

// device allocations and frees of a block of calls go to stream s
struct AllocOn {
    cih_basis &b;
    cudaStream_t old;
    AllocOn(cih_basis &b_, cudaStream_t s) : b(b_), old(b_.stream) { b.stream = s; }
    ~AllocOn() { b.stream = old; }
};

}  // namespace

int upload_and_build_neighbours(cih_basis &b, cudaStream_t st, const std::function<int()> &host_rest)
{
    int rc;
    const int W = b.W;
    b.stream = st;
    if ((rc = device_pool(b.device, &b.pool))) return rc;
    Timer tm("basis device set-up");
    if ((rc = dev_alloc(b, &b.dev_status, 4))) return rc;
    b.dev.queue = b.dev_status + 1;
    if (cudaMemsetAsync(b.dev_status, 0, 4 * sizeof(int), st) != cudaSuccess) return cuda_fail(cudaGetLastError(), "status");
    PinnedTotals pin;
    pin.st = st;
    cudaError_t e = pin.get();
    if (e != cudaSuccess) return cuda_fail(e, "pinned totals");
    for (int i = 0; i < 8; ++i) pin.p[i] = 0;
    Lists L[2];
    L[0].tot = pin.p;
    L[1].tot = pin.p + 3;
    // every kernel reads W words per bit string: they must hold every orbital
    for (int t = 0; t < 2; ++t)
        if (64 * W < b.s[t].n_orb || (W != 1 && W != 2 && W != 4))
            return fail(CIH_ERR_UNSUPPORTED, "internal: bit strings of " + std::to_string(W) + " words for " +
                                                 std::to_string(b.s[t].n_orb) + " orbitals");
    // 1. per species, protons on st and neutrons on a second stream: upload,
    //    hash table, staged passes (queued, no synchronisation).  Uploads from
    //    pageable memory wait for their own stream only, so neither species'
    //    uploads wait for the other's kernels.
    SpeciesHost H[2];
    side_by_side([&]() { species_prep(b, 0, H[0]); }, [&]() { species_prep(b, 1, H[1]); });
    SideStream side;
    if ((e = side.create()) != cudaSuccess) return cuda_fail(e, "side stream");
    const cudaStream_t ss[2] = {st, side.s};
    cudaEventRecord(side.ev[0], st);                   // after the status words are cleared
    cudaStreamWaitEvent(side.s, side.ev[0], 0);
    tm.mark("species host arrays");
    for (int t = 0; t < 2; ++t) {
        AllocOn on(b, ss[t]);
        if ((rc = species_upload(b, t, H[t], ss[t]))) return rc;
        if (W == 1) rc = lists_phase1<1>(b, t, b.sbuild[t], L[t], ss[t]);
        else if (W == 2) rc = lists_phase1<2>(b, t, b.sbuild[t], L[t], ss[t]);
        else rc = lists_phase1<4>(b, t, b.sbuild[t], L[t], ss[t]);
        if (rc) return rc;
    }
    tm.mark("species queued");
    // host work that the kernels above do not need: ranges, table layout, pn split
    if ((rc = host_rest())) return rc;
    tm.mark("host ranges + layout");
    e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(side.s);
    if (e != cudaSuccess) return cuda_fail(e, "neighbour counts");
    tm.mark("staged passes done");
    // basis tables while both streams are idle (no upload waits for a kernel)
    if ((rc = basis_tables_upload(b, st)) || (rc = upload(b, &L[1].rn, b.pn.rn, st))) return rc;
    cudaEventRecord(side.ev[1], st);
    // 2. exact-size lists, 3. two-move indices and neutron move information,
    //    again one species per stream; phase 3 reads the basis tables
    for (int t = 0; t < 2; ++t) {
        AllocOn on(b, ss[t]);
        if ((rc = lists_phase2(b, t, b.sbuild[t], L[t], ss[t]))) return rc;
        if (t == 1) cudaStreamWaitEvent(side.s, side.ev[1], 0);
        if (W == 1) rc = lists_phase3<1>(b, t, b.sbuild[t], L[t], ss[t]);
        else if (W == 2) rc = lists_phase3<2>(b, t, b.sbuild[t], L[t], ss[t]);
        else rc = lists_phase3<4>(b, t, b.sbuild[t], L[t], ss[t]);
        if (rc) return rc;
    }
    b.scan_scratch_len = scan_scratch_needed(b.dim);
    if ((rc = dev_alloc(b, &b.scan_scratch, b.scan_scratch_len))) return rc;
    {
        // neutron one-move lists: packed entries and bucket directory, and the
        // neutron occupied lists, on the second stream; the proton occupied
        // lists, candidate table and count lists (which read none of these) on st
        const Species &Q = b.s[1];
        int dm = 0;
        for (int x = 0; x < Q.n_orb; ++x)
            for (int y = 0; y < Q.n_orb; ++y) dm = std::max(dm, std::abs(Q.om2[x] - Q.om2[y]));
        const int NL = Q.Nsub_max + 1, RC = (dm + 1) * 2;
        const int dir_len = 1 + RC * NL;
        if (dir_len > 65535) return fail(CIH_ERR_UNSUPPORTED, "neutron bucket directory too long");
        const int64_t nn = Q.n_sd;
        const int64_t tot = L[1].tot[1];
        int2 *n1p;
        int16_t *dir, *srel;
        uint8_t *occp, *occn;
        const int g0 = (int)std::min<int64_t>((b.s[0].n_sd + 255) / 256 + 1, 65535);
        const int g1 = (int)std::min<int64_t>((nn + 255) / 256 + 1, 65535);
        {
            AllocOn on(b, side.s);
            if ((rc = dev_alloc(b, &n1p, tot)) || (rc = dev_alloc(b, &dir, (size_t)nn * dir_len)) ||
                (rc = dev_alloc(b, &srel, nn)) || (rc = dev_alloc(b, &occn, (size_t)nn * std::max(Q.Z, 1))))
                return rc;
            if (nn > 0) {
                count_launches(2);
                k_n1_pack<<<(int)std::min<int64_t>((tot + 255) / 256 + 1, 65535), 256, 0, side.s>>>(
                    nn, b.dev.sp[1].n1_off, b.dev.sp[1].n1, b.dev.n1_info, n1p);
                k_dir<<<grid_for(nn), 256, 0, side.s>>>(b.sbuild[1], b.dev.sp[1].n1_off, b.dev.sp[1].n1, NL, dm,
                                                        dir_len, dir);
            }
            count_launches(1);
            if (W == 1) k_occ<1><<<g1, 256, 0, side.s>>>(b.sbuild[1], Q.Z, b.dev.sp[1].n1_off, b.dev.sp[1].n1, occn, srel);
            else if (W == 2) k_occ<2><<<g1, 256, 0, side.s>>>(b.sbuild[1], Q.Z, b.dev.sp[1].n1_off, b.dev.sp[1].n1, occn, srel);
            else k_occ<4><<<g1, 256, 0, side.s>>>(b.sbuild[1], Q.Z, b.dev.sp[1].n1_off, b.dev.sp[1].n1, occn, srel);
        }
        cudaEventRecord(side.ev[2], side.s);           // the neutron half is complete here
        if ((rc = dev_alloc(b, &occp, (size_t)b.s[0].n_sd * std::max(b.s[0].Z, 1)))) return rc;
        count_launches(1);
        if (W == 1) k_occ<1><<<g0, 256, 0, st>>>(b.sbuild[0], b.s[0].Z, nullptr, nullptr, occp, nullptr);
        else if (W == 2) k_occ<2><<<g0, 256, 0, st>>>(b.sbuild[0], b.s[0].Z, nullptr, nullptr, occp, nullptr);
        else k_occ<4><<<g0, 256, 0, st>>>(b.sbuild[0], b.s[0].Z, nullptr, nullptr, occp, nullptr);
        b.dev.self_rel = srel;
        b.dev.occ[0] = occp;
        b.dev.occ[1] = occn;
        b.dev.n1p = n1p;
        b.dev.dir = dir;
        b.dev.dir_len = dir_len;
        b.dev.NL = NL;
        b.dev.DM = dm;
    }
    tm.mark("directory + occupied lists queued");
    {
        const int64_t np = b.s[0].n_sd;
        int64_t *coff;
        int32_t *row_p;
        if ((rc = dev_alloc(b, &coff, np + 1)) || (rc = dev_alloc(b, &row_p, b.dim))) return rc;
        int grid = grid_for(np);
        if (np > 0) {
            count_launches(1);
            k_cand_count<<<grid, 256, 0, st>>>(np, b.dev.sp[0].fw_off, b.dev.sp[0].n1_off, b.dev.sp[0].n1_later, coff);
        }
        if ((rc = exclusive_scan_i64(coff, np, b.scan_scratch, b.scan_scratch_len, st))) return rc;
        int64_t *total_p = pin.p + 6;
        e = cudaMemcpyAsync(total_p, coff + np, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "candidate count");
        const int64_t total = *total_p;
        int4 *cand;
        uint8_t *cself;
        if ((rc = dev_alloc(b, &cand, total)) || (rc = dev_alloc(b, &cself, total))) return rc;
        if (np > 0) {
            count_launches(2);
            const SpeciesBuild &SB = b.sbuild[0];
            if (W == 1) k_cand<1><<<grid, 256, 0, st>>>(SB, b.dev, SB.N, SB.M2, b.Nlim, coff, cand, cself);
            else if (W == 2) k_cand<2><<<grid, 256, 0, st>>>(SB, b.dev, SB.N, SB.M2, b.Nlim, coff, cand, cself);
            else k_cand<4><<<grid, 256, 0, st>>>(SB, b.dev, SB.N, SB.M2, b.Nlim, coff, cand, cself);
            k_row_p<<<grid, 256, 0, st>>>(np, b.dev.rowbase, row_p);
        }
        tm.mark("candidate table queued");
        b.dev.cand_off = coff;
        b.dev.cand = cand;
        b.dev.cand_self = cself;
        b.dev.row_p = row_p;
        // count lists (the count pass then reads a handful of directory entries per row)
        b.dev.clist_off = nullptr;
        b.dev.clist = nullptr;
        b.dev.cself_sfx = nullptr;
        if (np > 0 && b.dev.dir_len <= kClistDirCap && b.dev.NL <= 63) {
            int64_t *clen, *cloff;
            uint16_t *sfx;
            if ((rc = dev_alloc(b, &clen, np + 1)) || (rc = dev_alloc(b, &sfx, (size_t)np * b.dev.NL))) return rc;
            const int wpb = 8;
            const size_t sh = (size_t)wpb * (b.dev.dir_len + 64) * sizeof(int);
            if ((e = cudaFuncSetAttribute(k_clists<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh)) != cudaSuccess ||
                (e = cudaFuncSetAttribute(k_clists<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh)) != cudaSuccess)
                return cuda_fail(e, "count lists shared memory");
            const int gcl = (int)std::min<int64_t>((np + wpb - 1) / wpb, 152 * 8);
            count_launches(1);
            k_clists<0><<<gcl, 32 * wpb, sh, st>>>(np, coff, cand, cself, b.dev.dir_len, b.dev.NL, clen, nullptr,
                                                   nullptr, nullptr);
            if ((rc = exclusive_scan_i64(clen, np, b.scan_scratch, b.scan_scratch_len, st))) return rc;
            cloff = clen;
            int64_t *ctot = pin.p + 7;
            e = cudaMemcpyAsync(ctot, cloff + np, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(e, "count list size");
            int2 *cl;
            if ((rc = dev_alloc(b, &cl, std::max<int64_t>(*ctot, 1)))) return rc;
            count_launches(1);
            k_clists<1><<<gcl, 32 * wpb, sh, st>>>(np, coff, cand, cself, b.dev.dir_len, b.dev.NL, nullptr, cloff,
                                                   cl, sfx);
            b.dev.clist_off = cloff;
            b.dev.clist = cl;
            b.dev.cself_sfx = sfx;
        }
        b.dev.A = b.space.Z + b.space.N;
        b.dev.nZ[0] = b.space.Z;
        b.dev.nZ[1] = b.space.N;
    }
    cudaStreamWaitEvent(st, side.ev[2], 0);            // join: later work on st sees both species
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "basis upload");
    b.dev.max_cand = (int32_t)L[0].tot[2];
    return CIH_OK;
}

}  // namespace cih

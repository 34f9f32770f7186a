// Count, fill and adjoint passes over the half-stored Hamiltonian.
//
// Sec. 4.1: the nonzeros are run through twice, once to count them so the
// arrays can be allocated, once to compute them; Sec. 2: only half of the
// symmetric matrix is generated and stored; Sec. 1: every element is
// independent of the others.
//
// Row i = (proton sub-det p, neutron sub-det n).  Its stored columns j >= i
// are walked in ascending order:
//   A. q = p: the diagonal, then n's forward same-class neighbours inside
//      p's partner range (neutron one- and two-moves);
//   B. q > p from p's forward same-class list (proton one- and two-moves)
//      followed by p's one-move neighbours in later classes; for each q the
//      neutron partners are n itself (if it lies in q's range) merged with
//      n's one-move neighbours inside q's range (two-moves of p need n_j = n).
// A warp owns a row; lanes take candidate proton sub-dets, find their
// neutron segment by binary search, and a warp scan places the segments.
//
// Matrix elements (bra = row i, ket = column j, R = orbitals common to both):
// the operator a+_a a+_b a_d a_c with a<b in the bra and c<d in the ket has
// the sign (-1)^(sum over x in {a,b,c,d} of #R below x); a one-move a <- c
// has the sign (-1)^(#R below a + #R below c) and sums V(ak, ck) over the
// spectators k in R in ascending combined order.  Proton and neutron moves
// of a pn element factorise (the cross-species counts cancel in pairs).
#include <algorithm>

#include "cih_internal.h"

namespace cih {
namespace {

constexpr int kWarpsPerBlock = 8;

template <int W>
__device__ __forceinline__ void ld_bits(const uint64_t *base, int64_t i, uint64_t (&o)[W])
{
#pragma unroll
    for (int w = 0; w < W; ++w) o[w] = base[i * W + w];
}

template <int W>
__device__ __forceinline__ int popc_xor(const uint64_t (&a)[W], const uint64_t (&b)[W])
{
    int c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += __popcll(a[w] ^ b[w]);
    return c;
}

// number of set bits of R strictly below bit k
template <int W>
__device__ __forceinline__ int below(const uint64_t (&R)[W], int k)
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

template <int W>
__device__ __forceinline__ int lowest_bit(const uint64_t (&x)[W])
{
#pragma unroll
    for (int w = 0; w < W; ++w)
        if (x[w]) return w * 64 + __ffsll((long long)x[w]) - 1;
    return -1;
}

template <int W>
__device__ __forceinline__ void clear_bit(uint64_t (&x)[W], int k) { x[k >> 6] &= ~(1ull << (k & 63)); }

// Table index of V(ab, cd) for combined orbitals in any order; false if the
// pairs are not one table entry (a bug in the walk: flagged by the caller).
__device__ __forceinline__ bool tbme_at(const DevBasis &B, int a, int b, int c, int d, int64_t &idx, int &sign)
{
    if ((unsigned)a >= (unsigned)B.ntot || (unsigned)b >= (unsigned)B.ntot ||
        (unsigned)c >= (unsigned)B.ntot || (unsigned)d >= (unsigned)B.ntot)
        return false;
    int32_t e1 = B.pid[a * B.ntot + b], e2 = B.pid[c * B.ntot + d];
    if (e1 < 0 || e2 < 0) return false;
    int g = (e1 >> 16) & 0xFFF;
    if (g != ((e2 >> 16) & 0xFFF)) return false;
    sign = (((e1 ^ e2) >> 30) & 1) ? -1 : 1;
    int64_t u = e1 & 0xFFFF, v = e2 & 0xFFFF;
    if (u > v) { int64_t t = u; u = v; v = t; }
    int64_t n = B.gsize[g];
    idx = B.goff[g] + u * n - u * (u - 1) / 2 + (v - u);
    return true;
}

enum Kind : int { kDiag = 0, kP1 = 1, kN1 = 2, kP2 = 3, kN2 = 4, kPN = 5 };

// Everything that identifies one matrix element's terms.
template <int W>
struct Elem {
    int kind;
    int sign;                 // sign of the whole two-body part
    int a, b, c, d;           // combined orbitals: a(,b) bra-only, c(,d) ket-only
    uint64_t rp[W], rn[W];    // spectators: common protons / neutrons
};

// Visit the two-body terms (table index, sign) of an element in the fixed
// order the values are summed in.
template <int W, class F>
__device__ __forceinline__ bool for_terms(const DevBasis &B, const Elem<W> &e, F &&f)
{
    int64_t idx;
    int s;
    const int nbase = B.sp[1].orb_base;
    switch (e.kind) {
    case kP2:
    case kN2:
    case kPN:
        if (!tbme_at(B, e.a, e.b, e.c, e.d, idx, s)) return false;
        f(idx, s * e.sign);
        return true;
    case kP1:
    case kN1: {
        // spectators ascending in combined order: protons, then neutrons
        for (int sp = 0; sp < 2; ++sp) {
            const uint64_t *R = sp == 0 ? e.rp : e.rn;
            int off = sp == 0 ? 0 : nbase;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                uint64_t m = R[w];
                while (m) {
                    int k = off + w * 64 + __ffsll((long long)m) - 1;
                    m &= m - 1;
                    if (!tbme_at(B, e.a, k, e.c, k, idx, s)) return false;
                    f(idx, s * e.sign);
                }
            }
        }
        return true;
    }
    default: {  // diagonal: all occupied pairs a<b, lexicographic
        for (int sa = 0; sa < 2; ++sa) {
            const uint64_t *Ra = sa == 0 ? e.rp : e.rn;
            int offa = sa == 0 ? 0 : nbase;
            for (int wa = 0; wa < W; ++wa) {
                uint64_t ma = Ra[wa];
                while (ma) {
                    int ka = wa * 64 + __ffsll((long long)ma) - 1;
                    ma &= ma - 1;
                    int A = offa + ka;
                    for (int sb = sa; sb < 2; ++sb) {
                        const uint64_t *Rb = sb == 0 ? e.rp : e.rn;
                        int offb = sb == 0 ? 0 : nbase;
                        for (int wb = 0; wb < W; ++wb) {
                            uint64_t mb = Rb[wb];
                            while (mb) {
                                int kb = wb * 64 + __ffsll((long long)mb) - 1;
                                mb &= mb - 1;
                                int Bc = offb + kb;
                                if (Bc <= A) continue;
                                if (!tbme_at(B, A, Bc, A, Bc, idx, s)) return false;
                                f(idx, s);
                            }
                        }
                    }
                }
            }
        }
        return true;
    }
    }
}

// ---------------------------------------------------------------- element set-up

template <int W>
__device__ __forceinline__ void make_diag(Elem<W> &e, const uint64_t (&pb)[W], const uint64_t (&nb)[W])
{
    e.kind = kDiag;
    e.sign = 1;
#pragma unroll
    for (int w = 0; w < W; ++w) { e.rp[w] = pb[w]; e.rn[w] = nb[w]; }
}

// one orbital moved within species `sp` (bra bits x, ket bits y), other species `o` unchanged
template <int W>
__device__ __forceinline__ void make_one(Elem<W> &e, int sp, int base, const uint64_t (&x)[W], const uint64_t (&y)[W],
                                         const uint64_t (&o)[W])
{
    uint64_t R[W], dx[W], dy[W];
#pragma unroll
    for (int w = 0; w < W; ++w) { R[w] = x[w] & y[w]; dx[w] = x[w] & ~y[w]; dy[w] = y[w] & ~x[w]; }
    int a = lowest_bit<W>(dx), c = lowest_bit<W>(dy);
    e.kind = sp == 0 ? kP1 : kN1;
    e.sign = ((below<W>(R, a) + below<W>(R, c)) & 1) ? -1 : 1;
    e.a = base + a;
    e.c = base + c;
#pragma unroll
    for (int w = 0; w < W; ++w) {
        e.rp[w] = sp == 0 ? R[w] : o[w];
        e.rn[w] = sp == 0 ? o[w] : R[w];
    }
}

// two orbitals moved within one species
template <int W>
__device__ __forceinline__ void make_two(Elem<W> &e, int sp, int base, const uint64_t (&x)[W], const uint64_t (&y)[W])
{
    uint64_t R[W], dx[W], dy[W];
#pragma unroll
    for (int w = 0; w < W; ++w) { R[w] = x[w] & y[w]; dx[w] = x[w] & ~y[w]; dy[w] = y[w] & ~x[w]; }
    int a = lowest_bit<W>(dx); clear_bit<W>(dx, a);
    int b = lowest_bit<W>(dx);
    int c = lowest_bit<W>(dy); clear_bit<W>(dy, c);
    int d = lowest_bit<W>(dy);
    e.kind = sp == 0 ? kP2 : kN2;
    e.sign = ((below<W>(R, a) + below<W>(R, b) + below<W>(R, c) + below<W>(R, d)) & 1) ? -1 : 1;
    e.a = base + a; e.b = base + b; e.c = base + c; e.d = base + d;
}

// one proton and one neutron moved
template <int W>
__device__ __forceinline__ void make_pn(Elem<W> &e, int nbase, const uint64_t (&px)[W], const uint64_t (&py)[W],
                                        const uint64_t (&nx)[W], const uint64_t (&ny)[W])
{
    uint64_t Rp[W], Rn[W], dpx[W], dpy[W], dnx[W], dny[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
        Rp[w] = px[w] & py[w]; dpx[w] = px[w] & ~py[w]; dpy[w] = py[w] & ~px[w];
        Rn[w] = nx[w] & ny[w]; dnx[w] = nx[w] & ~ny[w]; dny[w] = ny[w] & ~nx[w];
    }
    int a = lowest_bit<W>(dpx), c = lowest_bit<W>(dpy);
    int b = lowest_bit<W>(dnx), d = lowest_bit<W>(dny);
    e.kind = kPN;
    e.sign = ((below<W>(Rp, a) + below<W>(Rp, c) + below<W>(Rn, b) + below<W>(Rn, d)) & 1) ? -1 : 1;
    e.a = a; e.b = nbase + b; e.c = c; e.d = nbase + d;
}

// ---------------------------------------------------------------- the row walk

struct FillArgs {
    int K;
    double hw;
    const float *tbme;        // K x tbme_len
    const double *esp;        // combined orbital energies or null
    int32_t *col;
    float *val;               // K x nnz
    int64_t nnz;
};

struct GradArgs {
    int K;
    const double *psi;        // K x dim
    unsigned long long *acc;  // K x tbme_len fixed point
};

constexpr double kFixScale = 72057594037927936.0;   // 2^56

template <int W>
__device__ double one_body(const DevBasis &B, const FillArgs &F, const uint64_t (&pb)[W], const uint64_t (&nb)[W])
{
    double s = 0.0;
    for (int sp = 0; sp < 2; ++sp) {
        const uint64_t *R = sp == 0 ? pb : nb;
        int off = B.sp[sp].orb_base;
        for (int w = 0; w < W; ++w) {
            uint64_t m = R[w];
            while (m) {
                int k = off + w * 64 + __ffsll((long long)m) - 1;
                m &= m - 1;
                s += F.esp ? F.esp[k] : F.hw * ((double)B.orbN[k] + 1.5);
            }
        }
    }
    return s;
}

// Mode 0: count, 1: fill, 2: gradient
template <int W, int MODE>
__device__ __forceinline__ void emit(const DevBasis &B, const FillArgs &F, const GradArgs &G, int *status,
                                     int64_t pos, int64_t lim, int64_t row, int64_t colj, const Elem<W> &e,
                                     double diag1)
{
    if (MODE == 1) {
        if (pos >= lim) {                      // never for a consistent count: refuse the write
            atomicOr(status, 2);
            return;
        }
        F.col[pos] = (int32_t)colj;
        for (int k = 0; k < F.K; ++k) {
            const float *T = F.tbme + (int64_t)k * B.tbme_len;
            double s = e.kind == kDiag ? diag1 : 0.0;
            bool ok = for_terms<W>(B, e, [&](int64_t idx, int sg) { s += sg * (double)T[idx]; });
            if (!ok) atomicOr(status, 1);
            F.val[(int64_t)k * F.nnz + pos] = (float)s;
        }
    } else if (MODE == 2) {
        for (int k = 0; k < G.K; ++k) {
            const double *psi = G.psi + (int64_t)k * B.dim;
            double f = (colj == row ? 1.0 : 2.0) * psi[row] * psi[colj];
            unsigned long long *acc = G.acc + (int64_t)k * B.tbme_len;
            bool ok = for_terms<W>(B, e, [&](int64_t idx, int sg) {
                long long q = __double2ll_rn(sg * f * kFixScale);
                atomicAdd(acc + idx, (unsigned long long)q);
            });
            if (!ok) atomicOr(status, 1);
        }
    }
}

// first index in sorted list[lo, hi) whose value is >= key
__device__ __forceinline__ int64_t lower_bound(const int32_t *list, int64_t lo, int64_t hi, int32_t key)
{
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (list[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

template <int W, int MODE>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_walk(DevBasis B, const int64_t *rowptr, int64_t *counts, FillArgs F, GradArgs G, int *status)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const DevSpecies &SP = B.sp[0], &SN = B.sp[1];
    const int nbase = SN.orb_base;
    const unsigned lt = (1u << lane) - 1;

    if (MODE == 1) F.nnz = rowptr[B.dim];       // set stride of the values
    for (int64_t row = gw; row < B.dim; row += nw) {
        // proton sub-det of the row: last p with rowbase[p] <= row
        int lo = 0, hi = B.n_p - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (B.rowbase[mid] <= row) lo = mid; else hi = mid - 1;
        }
        const int p = lo;
        const int nbp = B.nb[p];
        const int n = nbp + (int)(row - B.rowbase[p]);
        const int nend = nbp + B.nc[p];
        uint64_t pb[W], nbits[W];
        ld_bits<W>(SP.bits, p, pb);
        ld_bits<W>(SN.bits, n, nbits);
        const int64_t out = MODE == 1 ? rowptr[row] : 0;
        const int64_t lim = MODE == 1 ? min(rowptr[row + 1], F.nnz) : 0;
        int64_t pos = 0;
        double diag1 = 0.0;
        if (MODE == 1) diag1 = one_body<W>(B, F, pb, nbits);

        // ---- A: diagonal, then same-class forward neutron neighbours in p's range
        if (lane == 0 && MODE != 0) {
            Elem<W> e;
            make_diag<W>(e, pb, nbits);
            emit<W, MODE>(B, F, G, status, out, lim, row, row, e, diag1);
        }
        pos = 1;
        {
            const int64_t f0 = SN.fw_off[n], f1 = SN.fw_off[n + 1];
            for (int64_t t0 = f0; t0 < f1; t0 += 32) {
                int64_t t = t0 + lane;
                int y = t < f1 ? SN.fw[t] : INT32_MAX;
                bool in = y < nend;
                unsigned m = __ballot_sync(0xffffffffu, in);
                if (MODE != 0 && in) {
                    uint64_t yb[W];
                    ld_bits<W>(SN.bits, y, yb);
                    Elem<W> e;
                    if (popc_xor<W>(nbits, yb) == 2) make_one<W>(e, 1, nbase, nbits, yb, pb);
                    else make_two<W>(e, 1, nbase, nbits, yb);
                    emit<W, MODE>(B, F, G, status, out + pos + __popc(m & lt), lim, row,
                                  B.rowbase[p] + (y - nbp), e, diag1);
                }
                pos += __popc(m);
                if (m != 0xffffffffu) break;          // sorted: nothing later is < nend
            }
        }

        // ---- B: later proton sub-dets
        const int64_t n1a = SN.n1_off[n], n1b = SN.n1_off[n + 1];
        const int64_t self_ins = lower_bound(SN.n1, n1a, n1b, n);   // where n sorts among its neighbours
        for (int list = 0; list < 2; ++list) {
            int64_t c0, c1;
            if (list == 0) {
                c0 = SP.fw_off[p]; c1 = SP.fw_off[p + 1];
            } else {
                c1 = SP.n1_off[p + 1];
                c0 = lower_bound(SP.n1, SP.n1_off[p], c1, SP.cls_end[p]);
            }
            const int32_t *cand = list == 0 ? SP.fw : SP.n1;
            for (int64_t k0 = c0; k0 < c1; k0 += 32) {
                int64_t k = k0 + lane;
                int q = -1, dp = 0;
                int64_t lo1 = 0, hi1 = 0;
                bool self = false;
                int len = 0;
                uint64_t qb[W];
                if (k < c1) {
                    q = cand[k];
                    ld_bits<W>(SP.bits, q, qb);
                    dp = popc_xor<W>(pb, qb) >> 1;
                    const int qb0 = B.nb[q], qb1 = qb0 + B.nc[q];
                    self = n >= qb0 && n < qb1;
                    if (dp == 2) {
                        len = self ? 1 : 0;
                    } else {
                        lo1 = lower_bound(SN.n1, n1a, n1b, qb0);
                        hi1 = lower_bound(SN.n1, lo1, n1b, qb1);
                        len = (int)(hi1 - lo1) + (self ? 1 : 0);
                    }
                }
                // warp exclusive scan of len
                int inc = len;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    int o = __shfl_up_sync(0xffffffffu, inc, d);
                    if (lane >= d) inc += o;
                }
                const int tot = __shfl_sync(0xffffffffu, inc, 31);
                if (MODE != 0 && len > 0) {
                    int64_t o = out + pos + (inc - len);
                    const int64_t cbase = B.rowbase[q] - B.nb[q];
                    if (dp == 2) {
                        Elem<W> e;
                        make_two<W>(e, 0, 0, pb, qb);
                        emit<W, MODE>(B, F, G, status, o, lim, row, cbase + n, e, diag1);
                    } else {
                        const int64_t ins = self ? (min(max(self_ins, lo1), hi1) - lo1) : -1;
                        for (int t = 0; t < len; ++t) {
                            Elem<W> e;
                            int nj;
                            if (t == ins) {
                                nj = n;
                                make_one<W>(e, 0, 0, pb, qb, nbits);
                            } else {
                                nj = SN.n1[lo1 + t - ((ins >= 0 && t > ins) ? 1 : 0)];
                                uint64_t yb[W];
                                ld_bits<W>(SN.bits, nj, yb);
                                make_pn<W>(e, nbase, pb, qb, nbits, yb);
                            }
                            emit<W, MODE>(B, F, G, status, o + t, lim, row, cbase + nj, e, diag1);
                        }
                    }
                }
                pos += tot;
            }
        }
        if (MODE == 0 && lane == 0) counts[row] = pos;
    }
}

int grid_rows(int64_t rows)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (rows + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sms * 32));
}

template <int MODE>
int launch_walk(const cih_basis &b, const int64_t *rowptr, int64_t *counts, const FillArgs &F,
                const GradArgs &G, cudaStream_t st)
{
    if (b.dim == 0) return CIH_OK;
    int grid = grid_rows(b.dim);
    dim3 blk(kWarpsPerBlock * 32);
    count_launches(1);
    if (b.W == 1) k_walk<1, MODE><<<grid, blk, 0, st>>>(b.dev, rowptr, counts, F, G, b.dev_status);
    else if (b.W == 2) k_walk<2, MODE><<<grid, blk, 0, st>>>(b.dev, rowptr, counts, F, G, b.dev_status);
    else k_walk<4, MODE><<<grid, blk, 0, st>>>(b.dev, rowptr, counts, F, G, b.dev_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "row walk launch");
    return CIH_OK;
}

__global__ void k_fix_to_double(int64_t n, const unsigned long long *acc, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)(long long)acc[i] / kFixScale;
}

}  // namespace

int launch_count(const cih_basis &b, int64_t *rowptr, cudaStream_t st)
{
    return launch_walk<0>(b, nullptr, rowptr, FillArgs{}, GradArgs{}, st);
}

int launch_scan(const cih_basis &b, int64_t *rowptr, cudaStream_t st)
{
    return exclusive_scan_i64(rowptr, b.dim, b.scan_scratch, b.scan_scratch_len, st);
}

int launch_fill(const cih_basis &b, const int64_t *rowptr, int K, double hw, const float *tbme,
                const double *esp, int32_t *col, float *val, cudaStream_t st)
{
    FillArgs F{K, hw, tbme, esp, col, val, 0};
    return launch_walk<1>(b, rowptr, nullptr, F, GradArgs{}, st);
}

int launch_grad(const cih_basis &b, const int64_t *rowptr, int K, const double *psi,
                unsigned long long *acc, cudaStream_t st)
{
    GradArgs G{K, psi, acc};
    return launch_walk<2>(b, rowptr, nullptr, FillArgs{}, G, st);
}

int launch_grad_finish(int64_t n, const unsigned long long *acc, double *grad, cudaStream_t st)
{
    if (n == 0) return CIH_OK;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, 65535);
    count_launches(1);
    k_fix_to_double<<<blocks, 256, 0, st>>>(n, acc, grad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gradient finish");
    return CIH_OK;
}

}  // namespace cih

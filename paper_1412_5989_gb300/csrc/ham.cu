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
// A warp owns a row; lanes take candidate proton sub-dets, read their
// neutron segment bounds from n's bucket directory, and a warp scan places
// the segments.  The count pass has a faster form that needs no walk
// (k_count_lists): per proton sub-det, the directory positions where its
// segments start and end, summed against n's directory.
//
// Matrix elements (bra = row i, ket = column j, R = orbitals common to both):
// the operator a+_a a+_b a_d a_c with a<b in the bra and c<d in the ket has
// the sign (-1)^(sum over x in {a,b,c,d} of #R below x); a one-move a <- c
// has the sign (-1)^(#R below a + #R below c) and sums V(ak, ck) over the
// spectators k in R in ascending combined order.  Proton and neutron moves
// of a pn element factorise (the cross-species counts cancel in pairs).
#include <algorithm>
#include <cstdlib>
#include <map>
#include <mutex>

#include "cih_internal.h"
#include "ham_common.cuh"

namespace cih {
namespace {

// What the fill writes and reads: K two-body sets, table entry t of set k at
// tbme[k * tb_sk + t * tb_si] (set-major: tb_sk = table length, tb_si = 1;
// interleaved: tb_sk = 1, tb_si = K).
struct FillArgs {
    int K;
    double hw;
    const float *tbme;
    int64_t tb_sk, tb_si;
    int vec4;                 // interleaved, K % 4 == 0, 16-byte aligned: float4 table reads (and
                              // float4 value writes when em)
    int em;                   // values element-major: val[e * K + k] (else set-major val[k * nnz + e])
    const double *esp;        // combined orbital energies or null
    int32_t *col;
    float *val;               // K x nnz
    int sharded;              // 1: col / val hold only the rows from shard_row on (positions
    int64_t shard_row;        //    relative to rowptr[shard_row], nnz = that shard's count)
    const double *t1;         // one-body table (OneBodyLayout) in place of the orbital energies, or null
};

// table index of t_ac for combined orbitals a, c (either order), -1 if they
// are not one group of the one-body layout
__device__ __forceinline__ int onebody_at(const DevBasis &B, int a, int c)
{
    const int g = B.ob_grp[a];
    if (g < 0 || g != B.ob_grp[c]) return -1;
    int u = B.ob_loc[a], v = B.ob_loc[c];
    if (u > v) { const int x = u; u = v; v = x; }
    const int n = B.ob_gsize[g];
    return B.ob_goff[g] + u * n - ((u * (u - 1)) >> 1) + (v - u);
}

// t_ac of a one-particle move as a double-float pair (zero without a one-body
// table); a pair outside the layout is flagged
__device__ __forceinline__ DF onebody_term(const DevBasis &B, const FillArgs &F, int a, int c, int *status)
{
    if (!F.t1) return df_of(0.f);
    const int k = onebody_at(B, a, c);
    if (k < 0) {
        atomicOr(status, 1);
        return df_of(0.f);
    }
    const double t = F.t1[k];
    const float hi = (float)t;
    return DF{hi, (float)(t - (double)hi)};
}

struct GradArgs {
    int K;
    const long long *psi;     // K x dim, psi_i * 2^61 rounded (|psi_i| < 4)
    unsigned long long *acc;  // K x tbme_len fixed point, 2^56 units
};

constexpr double kFixScale = 72057594037927936.0;   // 2^56
constexpr double kPsiScale = 2305843009213693952.0;  // 2^61

// psi_i psi_j in units of 2^-58: the high 64 bits of the 128-bit product of
// the two 2^61-scaled vectors (integer arithmetic, exact but for the floor)
__device__ __forceinline__ long long psi_prod(const long long *psi, int64_t i, int64_t j)
{
    return __mul64hi(psi[i], psi[j]);
}

// ---------------------------------------------------------------- row kernel
//
// Warps walk rows independently (grid-stride); a CTA only shares the pn
// split table S in shared memory.  For row (p, n):
//   diagonal  - the warp sums the one-body energies and every occupied pair
//               (lanes over pairs, double-float reduction);
//   A         - n's forward same-class neighbours inside p's partner range:
//               two-moves from their precomputed table index, one-moves
//               deferred;
//   B         - p's candidate records in chunks of 64, two per lane: a lane
//               reads its candidates' neutron segments from n's bucket
//               directory (plus n itself if inside q's range), a warp scan
//               places the segments and the chunk's pn elements are emitted
//               flattened (lane e writes element e: contiguous stores).  pp two-moves use the precomputed
//               index, pn elements u(a,b) = S[a][kappa] + r(b), proton
//               one-moves are deferred;
//   deferred  - one-move elements, lanes over (element, spectator) pairs and
//               a segmented double-float reduction (K sets: lanes over sets).

constexpr int kLaneSets = 16;     // from this many sets on, multi-term sums run with lanes over sets
constexpr int kSlowCap = 64;
constexpr int kMaxA = 64;
constexpr int kPairCap = kMaxA * (kMaxA - 1) / 2;

namespace sm {
constexpr int gsize = 0;                                   // int32[kGroupCap]
constexpr int goff = gsize + kGroupCap * 4;                // int32[kGroupCap]
constexpr int pi = goff + kGroupCap * 4;                   // uint8[kPairCap]
constexpr int pj = pi + kPairCap;                          // uint8[kPairCap]
constexpr int lg = (pj + kPairCap + 15) / 16 * 16;         // int2[kLayoutCap]: table group size, offset
constexpr int e1 = lg + kLayoutCap * 8;                    // float2[kOrbCap]: one-body energies, hi + lo
constexpr int warp0 = e1 + kOrbCap * 8;
// per warp
constexpr int w_seg = 0;                                   // int4[64]: colbase, uv, mv, row start
constexpr int w_ext = w_seg + 64 * 16;                     // int2[64]: list start, insertion point
constexpr int w_spos = w_ext + 64 * 8;                     // int32[kSlowCap]
constexpr int w_scol = w_spos + kSlowCap * 4;              // int32[kSlowCap]
constexpr int w_scode = w_scol + kSlowCap * 4;             // uint32[kSlowCap]
constexpr int w_occ = w_scode + kSlowCap * 4;              // int16[kMaxA], then int2[32]: spectator entries
constexpr int w_size = (w_occ + kMaxA * 2 + 32 * 8 + 15) / 16 * 16;
// the pn split table S (int16[n_orb_p * G]) follows the per-warp areas
template <int WARPS>
constexpr int S = warp0 + WARPS * w_size;
}  // namespace sm

template <int WARPS>
inline size_t smem_bytes(int nS) { return (size_t)sm::S<WARPS> + ((size_t)nS * 2 + 15) / 16 * 16; }

template <class T>
__device__ __forceinline__ T *sptr(unsigned char *base, int off) { return reinterpret_cast<T *>(base + off); }

__device__ __forceinline__ DF warp_sum(DF v, int width)
{
    for (int d = width >> 1; d > 0; d >>= 1) {
        const DF o{__shfl_xor_sync(0xffffffffu, v.hi, d, width), __shfl_xor_sync(0xffffffffu, v.lo, d, width)};
        v = df_add(v, o);
    }
    return v;
}

template <int WARPS>
__device__ __forceinline__ int pn_index(const unsigned char *sb, uint32_t uv, uint32_t mv, uint32_t ni, int &sign)
{
    return pn_index_at(reinterpret_cast<const int16_t *>(sb + sm::S<WARPS>),
                       reinterpret_cast<const int32_t *>(sb + sm::gsize),
                       reinterpret_cast<const int32_t *>(sb + sm::goff), uv, mv, ni, sign);
}

// Row output view: column and value pointers at the row's first element;
// the value of set k at row position e is val[e * es + k * ks].
struct RowOut {
    int32_t *col;
    float *val;
    int64_t es, ks;
    int64_t row;
    long long psir;           // adjoint with one vector: the row's own psi (2^-61 units)
};

// one single-term element (table index, sign bit) at row-relative position e
template <int MODE, bool K1>
__device__ __forceinline__ void put_single(const DevBasis &B, const FillArgs &F, const GradArgs &Gr, const RowOut &R,
                                           int e, int64_t colj, int idx, int sgn)
{
    if (MODE == 1) {
        __stcs(R.col + e, (int32_t)colj);                         // evict-first: the walk's tables stay in L2
        if (K1) {                                                // K = 1: stride 1 in either layout
            const float v = __ldg(F.tbme + idx);
            __stcs(R.val + e, sgn ? -v : v);
        } else {
            // K sets: the value of set k goes to val[e * es + k * ks]; the sign flips bit 31
            const float *t = F.tbme + (int64_t)idx * F.tb_si;
            const int sm = sgn ? (int)0x80000000 : 0;
            if (F.em) {                                          // the K values of e are contiguous
                float *o = R.val + (int64_t)e * R.es;
                if (F.vec4) {
                    const float4 *t4 = reinterpret_cast<const float4 *>(t);
                    float4 *o4 = reinterpret_cast<float4 *>(o);
#pragma unroll 4
                    for (int k4 = 0; k4 < (F.K >> 2); ++k4) {
                        float4 v = __ldg(t4 + k4);
                        v.x = __int_as_float(__float_as_int(v.x) ^ sm);
                        v.y = __int_as_float(__float_as_int(v.y) ^ sm);
                        v.z = __int_as_float(__float_as_int(v.z) ^ sm);
                        v.w = __int_as_float(__float_as_int(v.w) ^ sm);
                        o4[k4] = v;
                    }
                } else {
                    for (int k = 0; k < F.K; ++k) o[k] = __int_as_float(__float_as_int(__ldg(t + k * F.tb_sk)) ^ sm);
                }
                return;
            }
            float *out = R.val + e;
            const int64_t vs = R.ks;
            if (F.vec4) {                                        // the K values of idx are contiguous
                const float4 *t4 = reinterpret_cast<const float4 *>(t);
#pragma unroll 4
                for (int k4 = 0; k4 < (F.K >> 2); ++k4) {
                    const float4 v = __ldg(t4 + k4);
                    float *o = out + (int64_t)(4 * k4) * vs;
                    o[0] = __int_as_float(__float_as_int(v.x) ^ sm);
                    o[vs] = __int_as_float(__float_as_int(v.y) ^ sm);
                    o[2 * vs] = __int_as_float(__float_as_int(v.z) ^ sm);
                    o[3 * vs] = __int_as_float(__float_as_int(v.w) ^ sm);
                }
            } else {
                const int64_t sk = F.tb_sk;
                int k = 0;
                for (; k + 4 <= F.K; k += 4) {                   // four independent reads in flight
                    const float v0 = __ldg(t + k * sk), v1 = __ldg(t + (k + 1) * sk);
                    const float v2 = __ldg(t + (k + 2) * sk), v3 = __ldg(t + (k + 3) * sk);
                    float *o = out + (int64_t)k * vs;
                    o[0] = __int_as_float(__float_as_int(v0) ^ sm);
                    o[vs] = __int_as_float(__float_as_int(v1) ^ sm);
                    o[2 * vs] = __int_as_float(__float_as_int(v2) ^ sm);
                    o[3 * vs] = __int_as_float(__float_as_int(v3) ^ sm);
                }
                for (; k < F.K; ++k) out[(int64_t)k * vs] = __int_as_float(__float_as_int(__ldg(t + k * sk)) ^ sm);
            }
        }
    } else if (MODE == 2) {
        for (int k = 0; k < (K1 ? 1 : Gr.K); ++k) {             // w psi_i psi_j, w = 2: 2^-57 units
            const long long q = (K1 ? __mul64hi(R.psir, Gr.psi[colj]) : psi_prod(Gr.psi + (int64_t)k * B.dim, R.row, colj)) >> 1;
            atomicAdd(Gr.acc + (int64_t)k * B.tbme_len + idx, (unsigned long long)(sgn ? -q : q));
        }
    }
}

// Element-major K-set values of up to 32 single-term elements, one per lane
// (act, table index idx, sign bit sgn, row position e), written by the whole
// warp: K/4 lanes copy one element's K values as float4s, so that a store
// instruction covers whole lines.  Needs F.em, F.vec4 and K/4 dividing 32 or
// a multiple of 32.  Columns are written by the caller.
template <int KC>
__device__ __forceinline__ void put_values_coop(const FillArgs &F, const RowOut &R, bool act, int idx, int sgn, int e)
{
    const int KK = KC > 0 ? KC : F.K;                          // KC > 0: the set count at compile time
    const int lane = threadIdx.x & 31;
    const unsigned am = __ballot_sync(0xffffffffu, act);
    if (!am) return;
    const int L = KK >> 2;                                       // float4s per element
    const int last = 31 - __clz(am);
    if (L <= 32) {
        // four rounds of P elements at a time: the four table reads are in
        // flight together before their stores
        constexpr int kB = 4;
        const int P = 32 / L, sub = lane / L, q = lane % L;
        for (int j0 = 0; j0 <= last; j0 += kB * P) {
            float4 v[kB];
            int64_t at[kB];
            bool on[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int src = j0 + u * P + sub;
                const int jidx = __shfl_sync(0xffffffffu, idx, src & 31);
                const int je = __shfl_sync(0xffffffffu, e, src & 31);
                const int js = __shfl_sync(0xffffffffu, sgn, src & 31);
                on[u] = src < 32 && ((am >> (src & 31)) & 1);
                at[u] = (int64_t)je * R.es;
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (on[u]) {
                    const int sm = js ? (int)0x80000000 : 0;
                    v[u] = __ldg(reinterpret_cast<const float4 *>(F.tbme + (int64_t)jidx * KK) + q);
                    v[u].x = __int_as_float(__float_as_int(v[u].x) ^ sm);
                    v[u].y = __int_as_float(__float_as_int(v[u].y) ^ sm);
                    v[u].z = __int_as_float(__float_as_int(v[u].z) ^ sm);
                    v[u].w = __int_as_float(__float_as_int(v[u].w) ^ sm);
                }
            }
#pragma unroll
            for (int u = 0; u < kB; ++u)                          // evict-first: the tables stay in L2
                if (on[u]) __stcs(reinterpret_cast<float4 *>(R.val + at[u]) + q, v[u]);
        }
    } else {
        for (int j = 0; j <= last; ++j) {
            const int jidx = __shfl_sync(0xffffffffu, idx, j);
            const int je = __shfl_sync(0xffffffffu, e, j);
            const int js = __shfl_sync(0xffffffffu, sgn, j);
            if (!((am >> j) & 1)) continue;
            const int sm = js ? (int)0x80000000 : 0;
            const float4 *t4 = reinterpret_cast<const float4 *>(F.tbme + (int64_t)jidx * KK);
            float4 *o4 = reinterpret_cast<float4 *>(R.val + (int64_t)je * R.es);
            for (int q = lane; q < L; q += 32) {
                float4 v = __ldg(t4 + q);
                v.x = __int_as_float(__float_as_int(v.x) ^ sm);
                v.y = __int_as_float(__float_as_int(v.y) ^ sm);
                v.z = __int_as_float(__float_as_int(v.z) ^ sm);
                v.w = __int_as_float(__float_as_int(v.w) ^ sm);
                o4[q] = v;
            }
        }
    }
}

// Deferred one-move elements of a row: lanes over (element, spectator)
// pairs, groups of the next power of two >= A-1 lanes, segmented sum (from
// kLaneSets sets on: one element at a time, lanes over sets).
// The queue holds row-relative positions, columns and packed moves
// (bra-only a, ket-only c, sign, neutron flag in bit 31).
template <int MODE, bool K1, int EM>
__device__ __forceinline__ void flush_slow(const DevBasis &B, const int2 *lg, const FillArgs &F, const GradArgs &Gr,
                                           int *status, const int16_t *w_occ, const int32_t *w_spos,
                                           const int32_t *w_scol, const uint32_t *w_scode, int &nslow,
                                           const RowOut &R)
{
    const int lane = threadIdx.x & 31;
    const int A = B.A, nbase = B.sp[1].orb_base;
    __syncwarp();
    const int ns = nslow;
    const int sp_n = A - 1;
    if (MODE == 1 && !K1 && F.K >= kLaneSets) {
        // K sets: the table entries of 32 / (A - 1) elements at a time (lanes
        // over (element, spectator) pairs, so their lookups run together), then
        // per element lanes over sets sum them in spectator order
        int2 *spec = reinterpret_cast<int2 *>(const_cast<int16_t *>(w_occ) + kMaxA);
        const int per = sp_n > 0 ? 32 / sp_n : 32;
        for (int e0 = 0; e0 < ns; e0 += per) {
            {
                const int ei = sp_n > 0 ? lane / sp_n : lane, i = sp_n > 0 ? lane % sp_n : 0;
                const int e = e0 + ei;
                if (ei < per && e < ns && i < sp_n) {
                    const uint32_t code = w_scode[e];
                    const int base = (code >> 31) ? nbase : 0;
                    const int a = base + (int)(code & 0xFF), c = base + (int)((code >> 8) & 0xFF);
                    int ia = 0;
                    for (int x = 0; x < A; ++x) ia += (w_occ[x] < a);
                    const int kspec = w_occ[i + (i >= ia ? 1 : 0)];
                    int64_t idx = 0;
                    int sg = 1;
                    const bool ok = tbme_at(B, lg, a, kspec, c, kspec, idx, sg);
                    if (!ok && atomicOr(status, 1) == 0) {
                        status[2] = a | (c << 16);
                        status[3] = 2 | (kspec << 8);
                    }
                    spec[ei * sp_n + i] = make_int2(ok ? (int)idx : -1, sg);
                }
            }
            __syncwarp();
            const int ne = min(per, ns - e0);
            const int KK = EM > 1 ? EM : F.K;                 // EM > 1: the set count at compile time
            const int L4 = KK >> 2;
            if (EM) {
                // element-major values: K/4 lanes per element with float4 reads and
                // writes, 32 / (K/4) elements at a time; each set's sum in the same
                // order as below
                const int P = 32 / L4, sub = lane / L4, q4 = lane % L4;
                for (int j0 = 0; j0 < ne; j0 += P) {
                    const int j = j0 + sub;
                    if (j >= ne) continue;
                    const int e = e0 + j;
                    const uint32_t code = w_scode[e];
                    const int base = (code >> 31) ? nbase : 0;
                    const int a = base + (int)(code & 0xFF), c = base + (int)((code >> 8) & 0xFF);
                    const int sgn = (code >> 16) & 1;
                    const int eo = w_spos[e];
                    const DF t1v = onebody_term(B, F, a, c, status);
                    const int2 *sj = spec + j * sp_n;
                    DF v0 = t1v, v1 = t1v, v2 = t1v, v3 = t1v;
#pragma unroll 8
                    for (int i = 0; i < sp_n; ++i) {
                        const int2 q = sj[i];
                        if (q.x < 0) continue;
                        float4 t = __ldg(reinterpret_cast<const float4 *>(F.tbme + (int64_t)q.x * KK) + q4);
                        if (q.y < 0) { t.x = -t.x; t.y = -t.y; t.z = -t.z; t.w = -t.w; }
                        v0 = df_add(v0, df_of(t.x));
                        v1 = df_add(v1, df_of(t.y));
                        v2 = df_add(v2, df_of(t.z));
                        v3 = df_add(v3, df_of(t.w));
                    }
                    float4 r = make_float4(df_round(v0), df_round(v1), df_round(v2), df_round(v3));
                    if (sgn) { r.x = -r.x; r.y = -r.y; r.z = -r.z; r.w = -r.w; }
                    __stcs(reinterpret_cast<float4 *>(R.val + (int64_t)eo * R.es) + q4, r);
                    if (q4 == 0) R.col[eo] = w_scol[e];
                }
            }
            for (int j = 0; j < (EM ? 0 : ne); ++j) {                // the other layouts: one element at a time
                const int e = e0 + j;
                const uint32_t code = w_scode[e];
                const int base = (code >> 31) ? nbase : 0;
                const int a = base + (int)(code & 0xFF), c = base + (int)((code >> 8) & 0xFF);
                const int sgn = (code >> 16) & 1;
                const int eo = w_spos[e];
                const DF t1v = onebody_term(B, F, a, c, status);      // the one-body term first
                const int2 *sj = spec + j * sp_n;
                for (int k = lane; k < F.K; k += 32) {
                    DF v = t1v;
#pragma unroll 8
                    for (int i = 0; i < sp_n; ++i) {
                        const int2 q = sj[i];
                        if (q.x < 0) continue;
                        const float t = __ldg(F.tbme + (int64_t)k * F.tb_sk + (int64_t)q.x * F.tb_si);
                        v = df_add(v, df_of(q.y < 0 ? -t : t));
                    }
                    const float r = df_round(v);
                    R.val[(int64_t)eo * R.es + (int64_t)k * R.ks] = sgn ? -r : r;
                }
                if (lane == 0) R.col[eo] = w_scol[e];
            }
            __syncwarp();
        }
        nslow = 0;
        return;
    }
    int gsz = 1;
    while (gsz < sp_n) gsz <<= 1;
    const int per = 32 / gsz;
    for (int e0 = 0; e0 < ns; e0 += per) {
        const int e = e0 + lane / gsz;
        const int i = lane % gsz;
        const bool act = e < ns;
        const uint32_t code = act ? w_scode[e] : 0;
        const int base = (code >> 31) ? nbase : 0;
        const int a = base + (int)(code & 0xFF), c = base + (int)((code >> 8) & 0xFF);
        const int sgn = (code >> 16) & 1;
        int ia = 0;
        for (int x = 0; x < A; ++x) ia += (w_occ[x] < a);
        const bool has = act && i < sp_n;
        const int kspec = has ? w_occ[i + (i >= ia ? 1 : 0)] : 0;
        const int eo = act ? w_spos[e] : 0;
        const int64_t colj = act ? w_scol[e] : 0;
        int64_t idx = 0;
        int sg = 1;
        bool ok = true;
        if (has) ok = tbme_at(B, lg, a, kspec, c, kspec, idx, sg);
        if (!ok && atomicOr(status, 1) == 0) {
            status[2] = a | (c << 16);
            status[3] = 2 | (kspec << 8);
        }
        // the one-body term t_ac (one per element: added by its group's first lane)
        const DF t1v = (MODE == 1 && act && i == 0) ? onebody_term(B, F, a, c, status) : df_of(0.f);
        for (int kk = 0; kk < (K1 ? 1 : MODE == 1 ? F.K : Gr.K); ++kk) {
            if (MODE == 1) {
                DF v = df_of(0.f);
                if (has && ok) {
                    const float t = __ldg(F.tbme + (int64_t)kk * F.tb_sk + idx * F.tb_si);
                    v = df_of(sg < 0 ? -t : t);
                }
                v = df_add(t1v, v);
                v = warp_sum(v, gsz);
                if (act && i == 0) {
                    if (kk == 0) R.col[eo] = (int32_t)colj;
                    const float r = df_round(v);
                    R.val[(int64_t)eo * R.es + (int64_t)kk * R.ks] = sgn ? -r : r;
                }
            } else if (has && ok) {
                const long long q =
                    (K1 ? __mul64hi(R.psir, Gr.psi[colj]) : psi_prod(Gr.psi + (int64_t)kk * B.dim, R.row, colj)) >> 1;
                const bool neg = (sgn != 0) != (sg < 0);
                atomicAdd(Gr.acc + (int64_t)kk * B.tbme_len + idx, (unsigned long long)(neg ? -q : q));
            }
        }
    }
    __syncwarp();
    nslow = 0;
}

template <int W, int MODE, bool K1, int WARPS, int EM>
__global__ void __launch_bounds__(WARPS * 32, 32 / WARPS)
k_rows(DevBasis B, const int64_t *rowptr, int64_t *counts, FillArgs F, GradArgs Gr, int64_t r0, int64_t r1,
       int *status)
{
    constexpr int kThreads = WARPS * 32;
    extern __shared__ __align__(16) unsigned char sb[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lt = (1u << lane) - 1;
    const DevSpecies &SP = B.sp[0], &SN = B.sp[1];
    const int A = B.A, nbase = SN.orb_base;
    const int npairs = A * (A - 1) / 2;
    if (MODE != 0) {
        const int G = B.pn_G, nS = SP.n_orb * G;
        int16_t *S = sptr<int16_t>(sb, sm::S<WARPS>);
        int32_t *gs = sptr<int32_t>(sb, sm::gsize), *go = sptr<int32_t>(sb, sm::goff);
        for (int i = tid; i < nS; i += kThreads) S[i] = B.pn_S[i];
        for (int i = tid; i < G; i += kThreads) { gs[i] = B.pn_gsize[i]; go[i] = B.pn_goff[i]; }
        if (B.ngroups <= kLayoutCap) {
            int2 *lgw = sptr<int2>(sb, sm::lg);
            for (int g = tid; g < B.ngroups; g += kThreads) lgw[g] = make_int2(B.gsize[g], (int)B.goff[g]);
        }
        if (MODE == 1) {                                   // one-body energies as hi + lo pairs
            float2 *e1w = sptr<float2>(sb, sm::e1);
            for (int a = tid; a < B.ntot && a < kOrbCap; a += kThreads) {
                const int k1 = F.t1 ? onebody_at(B, a, a) : -1;
                const double e = F.t1 ? (k1 >= 0 ? F.t1[k1] : 0.0) : F.esp ? F.esp[a] : F.hw * ((double)B.orbN[a] + 1.5);
                const float hi = (float)e;
                e1w[a] = make_float2(hi, (float)(e - (double)hi));
            }
        }
        uint8_t *pi = sptr<uint8_t>(sb, sm::pi), *pj = sptr<uint8_t>(sb, sm::pj);
        for (int l = tid; l < npairs; l += kThreads) {     // pair l -> (i, j), i < j
            int i = 0, r = l;
            while (r >= A - 1 - i) { r -= A - 1 - i; ++i; }
            pi[l] = (uint8_t)i;
            pj[l] = (uint8_t)(i + 1 + r);
        }
        __syncthreads();
    }
    // stored nonzeros the output arrays hold, and the row pointer of their first element
    const int64_t sbase = (MODE == 1 && F.sharded) ? rowptr[F.shard_row] : 0;
    const int64_t nnz = MODE == 1 ? (F.sharded ? rowptr[r1] - sbase : rowptr[B.dim]) : 0;
    const int2 *lg = sptr<int2>(sb, sm::lg);
    unsigned char *wb = sb + sm::warp0 + wid * sm::w_size;
    int4 *w_seg = sptr<int4>(wb, sm::w_seg);
    int2 *w_ext = sptr<int2>(wb, sm::w_ext);
    int32_t *w_spos = sptr<int32_t>(wb, sm::w_spos), *w_scol = sptr<int32_t>(wb, sm::w_scol);
    uint32_t *w_scode = sptr<uint32_t>(wb, sm::w_scode);
    int16_t *w_occ = sptr<int16_t>(wb, sm::w_occ);
    const int64_t gw = (blockIdx.x * (int64_t)kThreads + tid) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kThreads) >> 5;
    const int Zpro = B.nZ[0], Zneu = B.nZ[1];
    // K sets, element-major values: warp-cooperative value writes
    // (EM: the launcher chose this instantiation because F.em, F.vec4 and
    // K/4 dividing 32 or a multiple of 32 hold; the other K-set layouts
    // compile without these paths, and these without theirs)
    constexpr bool coop = MODE == 1 && !K1 && EM;

    for (int64_t row = r0 + gw; row < r1; row += nw) {
        const int p = B.row_p[row];
        const int nbp = B.nb[p];
        const int64_t rbp = B.rowbase[p];
        const int n = nbp + (int)(row - rbp);
        const int nend = nbp + B.nc[p];
        const int64_t cbp = rbp - nbp;
        RowOut R;
        R.row = row;
        R.psir = (MODE == 2 && K1) ? Gr.psi[row] : 0;
        R.es = (MODE == 1 && F.em) ? (EM > 1 ? EM : F.K) : 1;
        R.ks = (MODE == 1 && F.em) ? 1 : nnz;
        int rowlen = 0;
        if (MODE == 1) {
            const int64_t r0 = rowptr[row] - sbase;
            rowlen = (int)(min(rowptr[row + 1] - sbase, nnz) - r0);
            R.col = F.col + r0;
            R.val = F.val + r0 * R.es;
        }
        int nslow = 0;

        // ---- diagonal: occupied orbitals (combined, ascending), then all pairs
        if (MODE != 0) {
            for (int i = lane; i < A; i += 32)
                w_occ[i] = i < Zpro ? (int16_t)B.occ[0][(int64_t)p * Zpro + i]
                                    : (int16_t)(nbase + B.occ[1][(int64_t)n * Zneu + (i - Zpro)]);
            __syncwarp();
            const uint8_t *pi = sptr<uint8_t>(sb, sm::pi), *pj = sptr<uint8_t>(sb, sm::pj);
            const bool kset = MODE == 1 && !K1 && F.K >= kLaneSets && npairs <= kSlowCap;
            if (kset) {
                // K sets: the pairs' table entries in the (still empty) deferred
                // queue arrays, then lanes over sets sum them in pair order
                for (int l = lane; l < npairs; l += 32) {
                    const int a = w_occ[pi[l]], c = w_occ[pj[l]];
                    int64_t idx;
                    int sg;
                    const bool ok = tbme_at(B, lg, a, c, a, c, idx, sg);
                    if (!ok && atomicOr(status, 1) == 0) { status[2] = a | (c << 16); status[3] = 1; }
                    w_scol[l] = ok ? (int32_t)idx : -1;
                    w_scode[l] = sg < 0 ? 1u : 0u;
                }
                __syncwarp();
                DF one = df_of(0.f);
                const float2 *e1 = sptr<float2>(sb, sm::e1);
                for (int i = 0; i < A; ++i) {
                    const float2 q = e1[w_occ[i]];
                    one = df_add(one, DF{q.x, q.y});
                }
                const int KK = EM > 1 ? EM : F.K;
                const int L4 = KK >> 2;
                if (EM && L4 <= 32) {
                    // element-major values: four sets per lane, float4 reads, the same
                    // per-set order as below
                    for (int q4 = lane; q4 < L4; q4 += 32) {
                        DF a0 = df_of(0.f), a1 = a0, a2 = a0, a3 = a0;
#pragma unroll 4
                        for (int l = 0; l < npairs; ++l) {
                            const int32_t idx = w_scol[l];
                            if (idx < 0) continue;
                            float4 t = __ldg(reinterpret_cast<const float4 *>(F.tbme + (int64_t)idx * KK) + q4);
                            if (w_scode[l]) { t.x = -t.x; t.y = -t.y; t.z = -t.z; t.w = -t.w; }
                            a0 = df_add(a0, df_of(t.x));
                            a1 = df_add(a1, df_of(t.y));
                            a2 = df_add(a2, df_of(t.z));
                            a3 = df_add(a3, df_of(t.w));
                        }
                        if (rowlen > 0)
                            __stcs(reinterpret_cast<float4 *>(R.val) + q4,
                                   make_float4(df_round(df_add(a0, one)), df_round(df_add(a1, one)),
                                               df_round(df_add(a2, one)), df_round(df_add(a3, one))));
                    }
                }
                for (int k = lane; k < (EM && L4 <= 32 ? 0 : F.K); k += 32) {
                    DF acc = df_of(0.f);
#pragma unroll 4
                    for (int l = 0; l < npairs; ++l) {
                        const int32_t idx = w_scol[l];
                        if (idx < 0) continue;
                        const float v = __ldg(F.tbme + (int64_t)k * F.tb_sk + (int64_t)idx * F.tb_si);
                        acc = df_add(acc, df_of(w_scode[l] ? -v : v));
                    }
                    if (rowlen > 0) R.val[(int64_t)k * R.ks] = df_round(df_add(acc, one));
                }
                if (lane == 0 && rowlen > 0) R.col[0] = (int32_t)row;
                __syncwarp();
            }
            for (int k = 0; k < (kset ? 0 : K1 ? 1 : MODE == 1 ? F.K : Gr.K); ++k) {
                DF acc = df_of(0.f);
                for (int l = lane; l < npairs; l += 32) {
                    const int a = w_occ[pi[l]], c = w_occ[pj[l]];
                    int64_t idx;
                    int sg;
                    if (!tbme_at(B, lg, a, c, a, c, idx, sg)) {
                        if (atomicOr(status, 1) == 0) { status[2] = a | (c << 16); status[3] = 1; }
                        continue;
                    }
                    if (MODE == 1) {
                        const float v = __ldg(F.tbme + (int64_t)k * F.tb_sk + idx * F.tb_si);
                        acc = df_add(acc, df_of(sg < 0 ? -v : v));
                    } else {                                     // w = 1 on the diagonal
                        const long long q = psi_prod(Gr.psi + (int64_t)k * B.dim, row, row) >> 2;
                        atomicAdd(Gr.acc + (int64_t)k * B.tbme_len + idx, (unsigned long long)(sg < 0 ? -q : q));
                    }
                }
                if (MODE == 1) {
                    const float2 *e1 = sptr<float2>(sb, sm::e1);
                    for (int i = lane; i < A; i += 32) {
                        const float2 q = e1[w_occ[i]];
                        acc = df_add(acc, DF{q.x, q.y});
                    }
                    acc = warp_sum(acc, 32);
                    if (lane == 0 && rowlen > 0) {
                        if (k == 0) R.col[0] = (int32_t)row;
                        R.val[(int64_t)k * R.ks] = df_round(acc);
                    }
                }
            }
        }
        int pos = 1;

        // ---- A: same-class forward neutron neighbours inside p's range
        {
            const int64_t a0 = SN.fw_off[n], a1 = SN.fw_off[n + 1];
            for (int64_t t0 = a0; t0 < a1; t0 += 32) {
                const int64_t t = t0 + lane;
                const int y = t < a1 ? SN.fw[t] : INT32_MAX;
                const int32_t tbl = (MODE != 0 && t < a1) ? B.fw_tb[1][t] : 0;    // loaded beside y
                const bool in = y < nend;
                const unsigned bm = __ballot_sync(0xffffffffu, in);
                if (MODE != 0) {
                    if (MODE == 1 && pos + __popc(bm) > rowlen) { atomicOr(status, 2); break; }
                    if (nslow > kSlowCap - 32)
                        flush_slow<MODE, K1, EM>(B, lg, F, Gr, status, w_occ, w_spos, w_scol, w_scode, nslow, R);
                    const int32_t tb = in ? tbl : 0;
                    const bool slow = in && tb < 0;
                    const unsigned smk = __ballot_sync(0xffffffffu, slow);
                    const int e = pos + __popc(bm & lt);
                    if (MODE == 1 && coop) {
                        if (in && !slow) __stcs(R.col + e, (int32_t)(cbp + y));
                        put_values_coop<(EM > 1 ? EM : 0)>(F, R, in && !slow, tb >> 1, tb & 1, e);
                    } else if (in && !slow) {
                        put_single<MODE, K1>(B, F, Gr, R, e, cbp + y, tb >> 1, tb & 1);
                    }
                    if (slow) {
                        const int q = nslow + __popc(smk & lt);
                        w_spos[q] = e;
                        w_scol[q] = (int32_t)(cbp + y);
                        w_scode[q] = (uint32_t)~tb | (1u << 31);            // neutron one-move
                    }
                    nslow += __popc(smk);
                }
                pos += __popc(bm);
                if (bm != 0xffffffffu) break;
            }
        }

        // ---- B: candidates of p in chunks of 64, two per lane
        const int64_t c0 = B.cand_off[p], c1 = B.cand_off[p + 1];
        const int2 *n1row = B.n1p + SN.n1_off[n];
        const int16_t *dirn = B.dir + (int64_t)n * B.dir_len;
        const int Nn = SN.N[n];
        const int self_rel = B.self_rel[n];
        for (int64_t k0 = c0; k0 < c1; k0 += 64) {
            const bool v0 = k0 + 2 * lane < c1, v1 = k0 + 2 * lane + 1 < c1;
            int4 r0 = make_int4(0, 0, 0, 0), r1 = r0;
            int sl0 = 0, sl1 = 0;
            if (v0) { r0 = B.cand[k0 + 2 * lane]; sl0 = B.cand_self[k0 + 2 * lane]; }
            if (v1) { r1 = B.cand[k0 + 2 * lane + 1]; sl1 = B.cand_self[k0 + 2 * lane + 1]; }
            // each candidate: pn neutron moves [s_rel, s_rel + lpn) of n's list,
            // plus n itself (a pp two-move or a one-proton move) if inside q's range
            const bool self0 = (sl0 & 0x7F) > Nn, self1 = (sl1 & 0x7F) > Nn;   // 1 + L_q > N_n
            const int two0 = sl0 >> 7, two1 = sl1 >> 7;
            int lpn0 = 0, s0 = 0, lpn1 = 0, s1 = 0;
            if (v0 && !two0) { s0 = dirn[r0.y & 0xFFFF]; lpn0 = dirn[(unsigned)r0.y >> 16] - s0; }
            if (v1 && !two1) { s1 = dirn[r1.y & 0xFFFF]; lpn1 = dirn[(unsigned)r1.y >> 16] - s1; }
            const int lt0 = lpn0 + (self0 ? 1 : 0), lt1 = lpn1 + (self1 ? 1 : 0);
            // one scan of both counts (pn elements low half, all elements high half)
            const int pair = (lpn0 + lpn1) | ((lt0 + lt1) << 16);
            int incl = pair;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int o2 = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += o2;
            }
            const int tot = __shfl_sync(0xffffffffu, incl, 31);
            const int T = tot >> 16, Tpn = tot & 0xFFFF;
            if (MODE != 0 && T > 0) {
                if (MODE == 1 && pos + T > rowlen) { atomicOr(status, 2); pos += T; continue; }
                const int ex0 = pos + (incl >> 16) - (lt0 + lt1);        // row position of candidate 0
                const int ex1 = ex0 + lt0;
                const int ins0 = self0 && !two0 ? self_rel - s0 : -1;     // where n sorts among the pn moves
                const int ins1 = self1 && !two1 ? self_rel - s1 : -1;
                // n itself: written (pp two-move) or deferred (one-proton move) by its candidate's lane
                if (MODE == 1 && coop) {
                    if (self0 && two0) __stcs(R.col + ex0, r0.x + n);
                    if (self1 && two1) __stcs(R.col + ex1, r1.x + n);
                    put_values_coop<(EM > 1 ? EM : 0)>(F, R, self0 && two0, (int)((uint32_t)r0.z >> 1), r0.z & 1, ex0);
                    put_values_coop<(EM > 1 ? EM : 0)>(F, R, self1 && two1, (int)((uint32_t)r1.z >> 1), r1.z & 1, ex1);
                } else {
                    if (self0 && two0)
                        put_single<MODE, K1>(B, F, Gr, R, ex0, (int64_t)r0.x + n, (int)((uint32_t)r0.z >> 1), r0.z & 1);
                    if (self1 && two1)
                        put_single<MODE, K1>(B, F, Gr, R, ex1, (int64_t)r1.x + n, (int)((uint32_t)r1.z >> 1), r1.z & 1);
                }
                const bool p0 = self0 && !two0, p1 = self1 && !two1;
                const unsigned m0 = __ballot_sync(0xffffffffu, p0), m1 = __ballot_sync(0xffffffffu, p1);
                if (nslow + __popc(m0) + __popc(m1) > kSlowCap)
                    flush_slow<MODE, K1, EM>(B, lg, F, Gr, status, w_occ, w_spos, w_scol, w_scode, nslow, R);
                if (p0) {
                    const int q = nslow + __popc(m0 & lt);
                    const uint32_t mv = (uint32_t)r0.w;
                    w_spos[q] = ex0 + ins0;
                    w_scol[q] = r0.x + n;
                    w_scode[q] = ((mv >> 16) & 0xFF) | (((mv >> 24) & 0xFF) << 8) | (((mv >> 9) & 1) << 16);
                }
                nslow += __popc(m0);
                if (p1) {
                    const int q = nslow + __popc(m1 & lt);
                    const uint32_t mv = (uint32_t)r1.w;
                    w_spos[q] = ex1 + ins1;
                    w_scol[q] = r1.x + n;
                    w_scode[q] = ((mv >> 16) & 0xFF) | (((mv >> 24) & 0xFF) << 8) | (((mv >> 9) & 1) << 16);
                }
                nslow += __popc(m1);
                if (Tpn > 0) {
                    // compacted table of the chunk's non-empty pn segments: record, row
                    // position minus pn start, list start minus pn start, insertion point
                    const bool ne0 = lpn0 > 0, ne1 = lpn1 > 0;
                    const unsigned b0 = __ballot_sync(0xffffffffu, ne0), b1 = __ballot_sync(0xffffffffu, ne1);
                    const int q0 = __popc(b0 & lt) + __popc(b1 & lt), q1 = q0 + (ne0 ? 1 : 0);
                    const int incl_pn = incl & 0xFFFF;
                    const int st0 = incl_pn - lpn1 - lpn0, st1 = incl_pn - lpn1;     // pn starts
                    if (ne0) {
                        w_seg[q0] = make_int4(r0.x, r0.z, r0.w, ex0 - st0);
                        w_ext[q0] = make_int2(s0 - st0, ins0 >= 0 ? st0 + ins0 : INT32_MAX);
                    }
                    if (ne1) {
                        w_seg[q1] = make_int4(r1.x, r1.z, r1.w, ex1 - st1);
                        w_ext[q1] = make_int2(s1 - st1, ins1 >= 0 ? st1 + ins1 : INT32_MAX);
                    }
                    __syncwarp();
                    // element e belongs to the last non-empty segment starting at or
                    // before e: per 32-element window, a mask of the segment starts
                    // inside it (OR over lanes) and the count of earlier starts
                    const unsigned le = (2u << lane) - 1u;                 // bits 0..lane
                    int before = 0;                                        // segments started before the window
                    const int iters = (Tpn + 31) >> 5;
                    for (int it = 0; it < iters; ++it) {
                        const int w0 = it << 5;
                        unsigned mk = 0;
                        if (ne0 && st0 >= w0 && st0 < w0 + 32) mk |= 1u << (st0 - w0);
                        if (ne1 && st1 >= w0 && st1 < w0 + 32) mk |= 1u << (st1 - w0);
                        mk = __reduce_or_sync(0xffffffffu, mk);
                        const int e = w0 + lane;
                        int at = 0, idx = 0, sg = 0;
                        if (e < Tpn) {
                            const int j = before + __popc(mk & le) - 1;
                            const int4 sg4 = w_seg[j];
                            const int2 sx = w_ext[j];
                            at = sg4.w + e + (e >= sx.y ? 1 : 0);
                            const int2 ent = n1row[sx.x + e];
                            idx = pn_index<WARPS>(sb, (uint32_t)sg4.y, (uint32_t)sg4.z, (uint32_t)ent.y, sg);
                            if (MODE == 1 && coop) __stcs(R.col + at, sg4.x + ent.x);
                            else put_single<MODE, K1>(B, F, Gr, R, at, (int64_t)(sg4.x + ent.x), idx, sg);
                        }
                        if (MODE == 1 && coop) put_values_coop<(EM > 1 ? EM : 0)>(F, R, e < Tpn, idx, sg, at);
                        before += __popc(mk);
                    }
                    __syncwarp();
                }
            }
            pos += T;
        }
        if (MODE != 0 && nslow > 0) flush_slow<MODE, K1, EM>(B, lg, F, Gr, status, w_occ, w_spos, w_scol, w_scode, nslow, R);
        if (MODE == 0 && lane == 0) counts[row] = pos;
        __syncwarp();
    }
}

// Count pass from the count lists: for row (p, n), 1 for the diagonal + n's
// forward same-class neighbours inside p's range + the sum over p's list of
// coefficient x n's directory entry (the pn segment lengths of all of p's
// one-move candidates) + the candidates whose range holds n itself.  Equal to
// the walk's count, with no candidate records read.  Each row is a chain of
// dependent loads (row -> p -> n -> lists), so a warp takes 32 / G rows at a
// time, G lanes each, to keep that many chains in flight; every warp-wide
// intrinsic is reached by all 32 lanes.
template <int G>
__global__ void __launch_bounds__(256) k_count_lists(DevBasis B, int64_t *counts, int64_t r0, int64_t r1)
{
    constexpr int R = 32 / G;
    const int lane = threadIdx.x & 31, g = lane / G, li = lane % G;
    const unsigned full = 0xffffffffu, gbits = G == 32 ? full : (1u << G) - 1u;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const DevSpecies &SN = B.sp[1];
    for (int64_t base = r0 + gw * R; base < r1; base += nw * R) {      // uniform over the warp
        const int64_t row = base + g;
        const bool live = row < r1;
        int p = 0, n = 0, nend = 0;
        int64_t a0 = 0, a1 = 0, q0 = 0, q1 = 0;
        if (live) {
            p = B.row_p[row];
            const int nbp = B.nb[p];
            n = nbp + (int)(row - B.rowbase[p]);
            nend = nbp + B.nc[p];
            a0 = SN.fw_off[n];
            a1 = SN.fw_off[n + 1];
            q0 = B.clist_off[p];
            q1 = B.clist_off[p + 1];
        }
        // forward list, ascending: its entries below nend, G at a time
        int cnt = 0;
        bool more = live;
        for (int64_t t0 = a0; __any_sync(full, more); t0 += G) {
            const int64_t t = t0 + li;
            const bool in = more && t < a1 && SN.fw[t] < nend;
            const unsigned bm = (__ballot_sync(full, in) >> (g * G)) & gbits;
            if (more) {
                cnt += __popc(bm);
                more = bm == gbits;                    // the same in every lane of the group
            }
        }
        const int16_t *dirn = B.dir + (int64_t)n * B.dir_len;
        int acc = 0;
#pragma unroll 4
        for (int64_t q = q0 + li; q < q1; q += G) {
            const int2 e = B.clist[q];
            acc += e.y * (int)dirn[e.x];
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(full, acc, o);
        if (live && li == 0) counts[row] = 1 + cnt + acc + B.cself_sfx[(int64_t)p * B.NL + SN.N[n]];
    }
}

// Raise a kernel's dynamic shared-memory limit on a device once per size, so
// that later calls (inside a stream capture, say) only launch.
cudaError_t raise_smem_limit(const void *kern, int dev, int bytes)
{
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> raised;
    std::lock_guard<std::mutex> lock(mu);
    int &have = raised[{kern, dev}];
    if (bytes <= have) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

template <int MODE, int WARPS>
int launch_rows_w(const cih_basis &b, const int64_t *rowptr, int64_t *counts, const FillArgs &F, const GradArgs &G,
                  cudaStream_t st, bool dry, int64_t r0, int64_t r1)
{
    const DevBasis &D = b.dev;
    const size_t smem = MODE == 0 ? (size_t)sm::S<WARPS> : smem_bytes<WARPS>(D.sp[0].n_orb * D.pn_G);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto go = [&](auto kern) -> int {
        cudaError_t ee = raise_smem_limit((const void *)kern, dev, (int)smem);
        if (ee != cudaSuccess) return cuda_fail(ee, "row kernel shared memory");
        if (dry) return CIH_OK;                              // set-up only, no launch
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, smem);
        per_sm = std::max(per_sm, 1);
        if (b.launch_ctas > 0) per_sm = std::min(per_sm, b.launch_ctas);
        const int64_t want = (r1 - r0 + WARPS - 1) / WARPS;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * per_sm, want));
        count_launches(1);
        kern<<<grid, WARPS * 32, smem, st>>>(D, rowptr, counts, F, G, r0, r1, b.dev_status);
        ee = cudaGetLastError();
        return ee == cudaSuccess ? CIH_OK : cuda_fail(ee, "row kernel launch");
    };
    const bool k1 = (MODE == 1 && F.K == 1) || (MODE == 2 && G.K == 1);   // one set / one vector
    const int L4 = F.K >> 2;
    const bool em = MODE == 1 && !k1 && F.em && F.vec4 && (L4 > 32 ? L4 % 32 == 0 : 32 % L4 == 0);
    if constexpr (MODE == 1) {
        if (em) {                                            // element-major K sets: warp-cooperative writes
            if (F.K == 64) {                                 // the batched configuration's set count
                if (b.W == 1) return go(k_rows<1, MODE, false, WARPS, 64>);
                if (b.W == 2) return go(k_rows<2, MODE, false, WARPS, 64>);
                return go(k_rows<4, MODE, false, WARPS, 64>);
            }
            if (b.W == 1) return go(k_rows<1, MODE, false, WARPS, 1>);
            if (b.W == 2) return go(k_rows<2, MODE, false, WARPS, 1>);
            return go(k_rows<4, MODE, false, WARPS, 1>);
        }
    }
    if (b.W == 1) return k1 ? go(k_rows<1, MODE, true, WARPS, 0>) : go(k_rows<1, MODE, false, WARPS, 0>);
    if (b.W == 2) return k1 ? go(k_rows<2, MODE, true, WARPS, 0>) : go(k_rows<2, MODE, false, WARPS, 0>);
    return k1 ? go(k_rows<4, MODE, true, WARPS, 0>) : go(k_rows<4, MODE, false, WARPS, 0>);
}

template <int MODE>
int launch_rows(const cih_basis &b, const int64_t *rowptr, int64_t *counts, const FillArgs &F, const GradArgs &G,
                cudaStream_t st, bool dry = false, int64_t r0 = 0, int64_t r1 = -1)
{
    if (r1 < 0) r1 = b.dim;
    if (b.dim == 0 || (!dry && r1 <= r0)) return CIH_OK;
    const DevBasis &D = b.dev;
    if (D.pn_G > kGroupCap || D.A > kMaxA || D.A - 1 > 32)
        return fail(CIH_ERR_UNSUPPORTED, "more than 33 particles or pn groups above the row kernel's capacity");
    if (D.tbme_len > INT32_MAX) return fail(CIH_ERR_UNSUPPORTED, "two-body table above 2^31 entries");
    return b.launch_warps == 8 ? launch_rows_w<MODE, 8>(b, rowptr, counts, F, G, st, dry, r0, r1)
                               : launch_rows_w<MODE, 16>(b, rowptr, counts, F, G, st, dry, r0, r1);
}

// element-major copy of K set-major tables: out[t * K + k] = in[k * len + t]
__global__ void k_interleave(int K, int64_t len, const float *in, float *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len * K; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = i / K;
        const int k = (int)(i - t * K);
        out[i] = in[(int64_t)k * len + t];
    }
}

__global__ void k_fix_to_double(int64_t n, const unsigned long long *acc, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)(long long)acc[i] / kFixScale;
}

}  // namespace

int launch_count(const cih_basis &b, int64_t *rowptr, cudaStream_t st)
{
    if (!b.dev.clist_off || b.count_walk) return launch_rows<0>(b, nullptr, rowptr, FillArgs{}, GradArgs{}, st);
    if (b.dim == 0) return CIH_OK;
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    constexpr int G = 8;                                     // lanes per row
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_lists<G>, 256, 0);
    const int64_t rows_per_block = 8 * (32 / G);
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sms * std::max(per_sm, 1), (b.dim + rows_per_block - 1) / rows_per_block));
    count_launches(1);
    k_count_lists<G><<<grid, 256, 0, st>>>(b.dev, rowptr, 0, b.dim);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CIH_OK : cuda_fail(e, "count launch");
}

int launch_scan(const cih_basis &b, int64_t *rowptr, cudaStream_t st)
{
    return exclusive_scan_i64(rowptr, b.dim, b.scan_scratch, b.scan_scratch_len, st);
}

int launch_fill(const cih_basis &b, const int64_t *rowptr, int K, double hw, const float *tbme, bool interleaved,
                bool em, const double *esp, int32_t *col, float *val, cudaStream_t st, int64_t r0, int64_t r1,
                bool sharded, const double *t1)
{
    const int vec4 = interleaved && K % 4 == 0 && ((uintptr_t)tbme & 15) == 0 && (!em || ((uintptr_t)val & 15) == 0);
    FillArgs F{K, hw, tbme, interleaved ? 1 : b.layout.total, interleaved ? (int64_t)K : 1, vec4, em && K > 1 ? 1 : 0,
               esp, col, val, sharded ? 1 : 0, r0, t1};
    return launch_rows<1>(b, rowptr, nullptr, F, GradArgs{}, st, false, r0, r1);
}

int prepare_rows(const cih_basis &b, int K)
{
    FillArgs F{};
    F.K = K;
    GradArgs G{};
    G.K = K;
    int rc = launch_rows<0>(b, nullptr, nullptr, F, G, nullptr, true);
    if (!rc) rc = launch_rows<1>(b, nullptr, nullptr, F, G, nullptr, true);
    if (!rc) rc = launch_rows<2>(b, nullptr, nullptr, F, G, nullptr, true);
    return rc;
}

int launch_interleave(int K, int64_t len, const float *in, float *out, cudaStream_t st)
{
    if (len * K == 0) return CIH_OK;
    const int blocks = (int)std::min<int64_t>((len * K + 255) / 256, 152 * 16);
    count_launches(1);
    k_interleave<<<blocks, 256, 0, st>>>(K, len, in, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? CIH_OK : cuda_fail(e, "interleave");
}

// psi_fix[i] = psi[i] * 2^61 rounded; |psi| >= 4 cannot be held and sets status bit 32
__global__ void k_psi_fix(int64_t n, const double *psi, long long *psi_fix, int *status)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = psi[i];
        if (!(fabs(v) < 4.0)) {
            atomicOr(status, 32);
            psi_fix[i] = 0;
        } else {
            psi_fix[i] = __double2ll_rn(v * kPsiScale);
        }
    }
}

// ||psi_k||^2 of each set, one block per set: above 1 + 1e-6 sets status bit 32
// (|g_t| <= 2 ||psi||^2 must stay below the 2^7 the 2^-56 accumulators hold)
__global__ void __launch_bounds__(1024) k_psi_norm(int64_t dim, const double *psi, int *status)
{
    __shared__ double part[32];
    const double *v = psi + (int64_t)blockIdx.x * dim;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < dim; i += blockDim.x) s += v[i] * v[i];
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (threadIdx.x == 0 && !(s <= 1.0 + 1e-6)) atomicOr(status, 32);
    }
}

int launch_grad(const cih_basis &b, const int64_t *rowptr, int K, const double *psi,
                unsigned long long *acc, cudaStream_t st)
{
    const int64_t n = (int64_t)K * b.dim;
    if (n == 0) return CIH_OK;
    long long *fix = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&fix, sizeof(long long) * n, b.pool, st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(CIH_ERR_NOMEM, "adjoint: fixed-point vector");
    }
    count_launches(2);
    k_psi_norm<<<K, 1024, 0, st>>>(b.dim, psi, b.dev_status);
    k_psi_fix<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(n, psi, fix, b.dev_status);
    GradArgs G{K, fix, acc};
    const int rc = launch_rows<2>(b, rowptr, nullptr, FillArgs{}, G, st);
    cudaFreeAsync(fix, st);
    return rc;
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

// Host construction of the many-body basis and of the two-body table layout.
//
// Sec. 2 of the paper: the index tables that define the many-body basis are
// built before the Hamiltonian; Sec. 3.2: the single-particle quantum numbers
// are flattened into one linear orbital index.  The conventions are the
// ones stated in include/cih.h.
//
// Sub-determinants are generated directly in ascending bit-string order
// (colexicographic recursion over the highest occupied orbital) and then
// bucketed by (2M, parity, N) with a stable counting sort, which yields the
// (2M, N mod 2, N, bits) order in linear time.
#include <algorithm>
#include <tuple>
#include <memory>
#include <exception>
#include <thread>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <utility>

#include "cih_internal.h"

namespace cih {
namespace {

// Quanta of the lowest configuration of k particles of one species and the
// highest shell it touches (shell N holds (N+1)(N+2) states).
void lowest_configuration(int k, int &N0, int &NF)
{
    N0 = 0;
    NF = -1;
    for (int shell = 0; k > 0; ++shell) {
        int cap = (shell + 1) * (shell + 2);
        int take = std::min(k, cap);
        N0 += take * shell;
        k -= take;
        NF = shell;
    }
}

void make_orbitals(Species &s, int top_shell)
{
    s.oN.clear(); s.ol.clear(); s.oj2.clear(); s.om2.clear();
    for (int N = 0; N <= top_shell; ++N)
        for (int l = N & 1; l <= N; l += 2)
            for (int j2 = 2 * l - 1; j2 <= 2 * l + 1; j2 += 2) {
                if (j2 < 0) continue;
                for (int m2 = -j2; m2 <= j2; m2 += 2) {
                    s.oN.push_back(N); s.ol.push_back(l); s.oj2.push_back(j2); s.om2.push_back(m2);
                }
            }
    s.n_orb = (int)s.oN.size();
}

// Sub-determinants of one species in (2M, N mod 2, N, bits) order, in two
// passes over the highest occupied orbital `top`: pass 1 counts the subsets of
// each (top, bucket) with bucket = (2M, N mod 2, N), by a counting recursion
// over the orbitals rather than by enumeration; a prefix sum in (bucket, top)
// order gives each pair its slot; pass 2, in parallel over the tops,
// enumerates and writes every subset to its slot.  Inside one (top, bucket) the recursion visits subsets in
// ascending bit-string order (colexicographic: highest element first), and
// slots of the same bucket are ordered by top, so each bucket comes out
// sorted by the bit string read as an unsigned integer.
struct Enumerator {
    const Species &s;
    std::vector<int> minsum;      // quanta of the c lowest orbitals
    int Mabs = 0, nN = 0;

    explicit Enumerator(const Species &sp) : s(sp)
    {
        minsum.assign(s.Z + 1, 0);
        for (int c = 1; c <= s.Z; ++c) minsum[c] = minsum[c - 1] + s.oN[c - 1];
        std::vector<int> m(s.om2.begin(), s.om2.end());
        for (int &x : m) x = std::abs(x);
        std::sort(m.rbegin(), m.rend());
        for (int c = 0; c < s.Z && c < (int)m.size(); ++c) Mabs += m[c];
        nN = s.Nsub_max + 1;
    }
    // bucket key in (2M, N mod 2, N) order.  2M has the parity of Z (every 2m is
    // odd), as has Mabs, so (2M + Mabs) / 2 numbers the possible 2M values;
    // N maps to its rank among the even values, then the odd ones.
    int64_t nkeys() const { return (int64_t)(Mabs + 1) * nN; }
    int64_t key(int N, int M) const
    {
        const int r = (N & 1) ? (nN + 1) / 2 + (N >> 1) : (N >> 1);
        return (int64_t)((M + Mabs) >> 1) * nN + r;
    }

    // c more orbitals below `lim` with at most `budget` quanta; F(w, N, M) at each leaf
    template <class Fn>
    void rec(uint64_t *w, int c, int lim, int budget, int Nacc, int Macc, Fn &f) const
    {
        if (c == 0) { f(w, Nacc, Macc); return; }
        for (int a = c - 1; a < lim; ++a) {
            if (s.oN[a] + minsum[c - 1] > budget) break;     // orbitals sorted by N
            w[a >> 6] |= 1ull << (a & 63);
            rec(w, c - 1, a, budget - s.oN[a], Nacc + s.oN[a], Macc + s.om2[a], f);
            w[a >> 6] &= ~(1ull << (a & 63));
        }
    }
};

template <class Fn>
void parallel_tops(int ntop, Fn &&fn)
{
    unsigned hw = std::max(1u, std::min(4u, std::thread::hardware_concurrency()));
    if (const char *e = std::getenv("CIH_THREADS")) hw = (unsigned)std::max(1, std::atoi(e));
    int nt = (int)std::min<unsigned>(hw, (unsigned)std::max(ntop / 4, 1));
    if (nt <= 1) { for (int t = 0; t < ntop; ++t) fn(t); return; }
    std::vector<std::thread> th;
    for (int i = 0; i < nt; ++i)
        th.emplace_back([&, i]() { for (int t = i; t < ntop; t += nt) fn(t); });
    for (auto &x : th) x.join();
}

// The two passes of the enumeration, split so that the appearing filter can
// run between them: after both species' count passes, a bucket (2M, N) of
// one species appears when the other species has a non-empty bucket (2M',
// N') with 2M + 2M' = 2M_total, N + N' <= Nlim and N + N' = Nlim (mod 2) (the
// relation is symmetric, so the unfiltered counts decide it).  The write pass
// then gives slots to the appearing buckets only.
struct SubdetCount {
    std::unique_ptr<Enumerator> E;
    std::vector<int> tops;
    int64_t nk = 0;
    std::vector<int64_t> cnt;        // [top][bucket]
    std::vector<int64_t> total;      // per bucket
    int M2_of(int64_t k) const { return 2 * (int)(k / E->nN) - E->Mabs; }
    int N_of(int64_t k) const
    {
        const int r = (int)(k % E->nN), ne = (E->nN + 1) / 2;
        return r < ne ? 2 * r : 2 * (r - ne) + 1;
    }
};

void count_subdets(const Species &s, SubdetCount &C)
{
    if (s.Z == 0) return;                         // the empty sub-determinant: no passes
    Timer tm("enumerate");
    C.E.reset(new Enumerator(s));
    const Enumerator &E = *C.E;
    const int budget = s.Nsub_max;
    for (int a = s.Z - 1; a < s.n_orb; ++a)
        if (s.oN[a] + E.minsum[s.Z - 1] <= budget) C.tops.push_back(a);
    const int ntop = (int)C.tops.size();
    C.nk = E.nkeys();
    C.cnt.assign((size_t)ntop * C.nk, 0);          // one row per top
    // The counts need no enumeration: with the orbitals taken in index order,
    // T[c][N][2M] holds the number of c-subsets of the orbitals below the
    // current one with quanta N and projection 2M (a generating-function
    // recursion).  Top a's row is T[Z-1] shifted by a's own (N, 2M); then a is
    // added to every subset of fewer than Z-1 orbitals.  Since orbitals come in
    // ascending N, a c-subset below a still takes Z-c orbitals of at least N_a,
    // which bounds the useful N.
    const int Z = s.Z, NB = budget + 1, MS = 2 * E.Mabs + 1;
    std::vector<int64_t> T((size_t)Z * NB * MS, 0);
    auto row = [&](int c, int N) { return &T[((size_t)c * NB + N) * MS + E.Mabs]; };   // index by 2M
    row(0, 0)[0] = 1;
    int mreach = 0;                                // largest |2m| among the orbitals so far
    for (int a = 0, t = 0; a < s.n_orb && t < ntop; ++a) {
        const int Na = s.oN[a], ma = s.om2[a];
        mreach = std::max(mreach, std::abs(ma));
        if (a == C.tops[t]) {
            int64_t *cnt = &C.cnt[(size_t)t * C.nk];
            const int Mr = std::min(E.Mabs, (Z - 1) * mreach);
            for (int N = 0; N + Na <= budget; ++N) {
                const int64_t *r = row(Z - 1, N);
                for (int M = -Mr; M <= Mr; ++M)
                    if (r[M]) cnt[E.key(N + Na, M + ma)] += r[M];
            }
            ++t;
        }
        for (int c = std::min(Z - 2, a); c >= 0; --c) {
            const int Mr = std::min(E.Mabs, c * mreach);
            for (int N = 0; N + (Z - c) * Na <= budget; ++N) {
                const int64_t *r = row(c, N);
                int64_t *o = row(c + 1, N + Na) + ma;
                for (int M = -Mr; M <= Mr; ++M)
                    if (r[M]) o[M] += r[M];
            }
        }
    }
    C.total.assign(C.nk, 0);
    for (int t = 0; t < ntop; ++t)
        for (int64_t k = 0; k < C.nk; ++k) C.total[k] += C.cnt[(size_t)t * C.nk + k];
    tm.mark("count pass");
}

// (2M, N) of the non-empty buckets of a species (the empty sub-determinant
// when it has no particles)
std::vector<std::pair<int, int>> filled_buckets(const Species &s, const SubdetCount &C)
{
    std::vector<std::pair<int, int>> v;
    if (s.Z == 0) { v.push_back({0, 0}); return v; }
    for (int64_t k = 0; k < C.nk; ++k)
        if (C.total[k] > 0) v.push_back({C.M2_of(k), C.N_of(k)});
    return v;
}

// which (2M, N) of this species pair with some filled bucket of the other
bool appears(int M2, int N, int twoM, int Nlim, const std::vector<int> &minN, int mspan)
{
    const int room = Nlim - N, mo = twoM - M2;
    if (room < 0 || mo < -mspan || mo > mspan) return false;
    return minN[(size_t)(mo + mspan) * 2 + (room & 1)] <= room;
}

void write_subdets(Species &s, SubdetCount &C, const std::vector<char> &keep_key)
{
    if (s.Z == 0) {                               // the empty sub-determinant
        s.n_sd = keep_key.empty() || keep_key[0] ? 1 : 0;
        s.bits.assign((size_t)s.n_sd * kMaxWords, 0);
        s.N.assign(s.n_sd, 0);
        s.M2.assign(s.n_sd, 0);
        return;
    }
    Timer tm("enumerate");
    const Enumerator &E = *C.E;
    const int budget = s.Nsub_max;
    const int ntop = (int)C.tops.size();
    const int64_t nk = C.nk;
    // slots in (bucket, top) order over the kept buckets; a dropped bucket's
    // slots are -1 and its sub-determinants are not written
    std::vector<int64_t> run(nk, 0);
    int64_t total = 0;
    for (int64_t k = 0; k < nk; ++k) {
        run[k] = total;
        if (keep_key[k]) total += C.total[k];
    }
    for (int t = 0; t < ntop; ++t)
        for (int64_t k = 0; k < nk; ++k) {
            int64_t &c = C.cnt[(size_t)t * nk + k];
            const int64_t v = c;
            c = keep_key[k] ? run[k] : -1;
            run[k] += v;
        }
    tm.mark("prefix");
    s.n_sd = total;
    s.bits.assign((size_t)total * kMaxWords, 0);
    s.N.assign(total, 0);
    s.M2.assign(total, 0);
    parallel_tops(ntop, [&](int t) {
        uint64_t w[kMaxWords] = {0, 0, 0, 0};
        const int a = C.tops[t];
        w[a >> 6] |= 1ull << (a & 63);
        int64_t *slot = &C.cnt[(size_t)t * nk];
        auto f = [&](const uint64_t *wb, int N, int M) {
            int64_t &sl = slot[E.key(N, M)];
            if (sl < 0) return;
            const int64_t i = sl++;
            std::copy(wb, wb + kMaxWords, &s.bits[(size_t)i * kMaxWords]);
            s.N[i] = N;
            s.M2[i] = M;
        };
        E.rec(w, s.Z - 1, a, budget - s.oN[a], s.oN[a], s.om2[a], f);
    });
}



void make_classes(Species &s)
{
    s.cls.assign(s.n_sd, 0);
    s.cls_M2.clear(); s.cls_par.clear(); s.cls_begin.clear(); s.cls_end.clear();
    for (int64_t i = 0; i < s.n_sd; ++i) {
        if (i == 0 || s.M2[i] != s.M2[i - 1] || (s.N[i] & 1) != (s.N[i - 1] & 1)) {
            if (!s.cls_begin.empty()) s.cls_end.push_back((int)i);
            s.cls_M2.push_back(s.M2[i]);
            s.cls_par.push_back(s.N[i] & 1);
            s.cls_begin.push_back((int)i);
        }
        s.cls[i] = (int)s.cls_begin.size() - 1;
    }
    if (!s.cls_begin.empty()) s.cls_end.push_back((int)s.n_sd);
}

// Two-body table layout: see include/cih.h.
int build_layout(cih_basis &b)
{
    Layout &L = b.layout;
    const Species &P = b.s[0], &Nn = b.s[1];
    int ntot = P.n_orb + Nn.n_orb;
    L.pid.assign((size_t)ntot * ntot, -1);
    L.gsize.clear();
    L.goff.clear();
    auto orbN = [&](int a) { return a < P.n_orb ? P.oN[a] : Nn.oN[a - P.n_orb]; };
    auto orbM = [&](int a) { return a < P.n_orb ? P.om2[a] : Nn.om2[a - P.n_orb]; };
    int64_t base = 0;
    for (int c = 0; c < 3; ++c) {
        int need_p = c == 0 ? 2 : c == 1 ? 0 : 1;
        int need_n = c == 0 ? 0 : c == 1 ? 2 : 1;
        L.chan_len[c] = 0;
        if (P.Z < need_p || Nn.Z < need_n) continue;
        int a0, d0, a1, d1;
        lowest_configuration(P.Z - need_p, a0, d0);
        lowest_configuration(Nn.Z - need_n, a1, d1);
        int limit = b.Nlim - (a0 + a1);
        int alo = c == 1 ? P.n_orb : 0, ahi = c == 0 ? P.n_orb : (c == 1 ? ntot : P.n_orb);
        int blo = c == 0 ? 0 : P.n_orb, bhi = c == 0 ? P.n_orb : ntot;
        // groups keyed (2M_pair, parity), ascending: dense key (2M_pair + mspan) * 2 + parity
        int mspan = 0;
        for (int a = alo; a < ahi; ++a) mspan = std::max(mspan, std::abs(orbM(a)));
        for (int bb = blo; bb < bhi; ++bb) mspan = std::max(mspan, std::abs(orbM(bb)));
        mspan *= 2;
        std::vector<std::vector<std::pair<int, int>>> groups((size_t)(2 * mspan + 1) * 2);
        for (int a = alo; a < ahi; ++a)
            for (int bb = std::max(blo, a + 1); bb < bhi; ++bb)
                if (orbN(a) + orbN(bb) <= limit)
                    groups[(size_t)(orbM(a) + orbM(bb) + mspan) * 2 + ((orbN(a) + orbN(bb)) & 1)].push_back({a, bb});
        int64_t off = 0;
        for (auto &grp : groups) {
            if (grp.empty()) continue;
            int g = (int)L.gsize.size();
            int n = (int)grp.size();
            if (g >= (1 << 12) || n >= (1 << 16)) return fail(CIH_ERR_UNSUPPORTED, "table group too large");
            L.gsize.push_back(n);
            L.goff.push_back(base + off);
            for (int u = 0; u < n; ++u) {
                int a = grp[u].first, bb = grp[u].second;
                L.pid[(size_t)a * ntot + bb] = pair_code(g, u, false);
                L.pid[(size_t)bb * ntot + a] = pair_code(g, u, true);
            }
            off += (int64_t)n * (n + 1) / 2;
        }
        L.chan_len[c] = off;
        base += off;
    }
    L.total = base;
    return CIH_OK;
}

// u(a, b) = S[a][kappa] + r(b) for every pn pair of the table (see PnSplit);
// checked against the pair codes.
int build_pn_split(cih_basis &b)
{
    const Species &P = b.s[0], &Q = b.s[1];
    PnSplit &X = b.pn;
    int ntot = P.n_orb + Q.n_orb;
    // span covers every pn pair and every single orbital, so that the shifted
    // 2m_a + span of a proton orbital is never negative
    int span = 0;
    for (int a = 0; a < P.n_orb; ++a) span = std::max(span, std::abs(P.om2[a]));
    for (int c = 0; c < Q.n_orb; ++c) span = std::max(span, std::abs(Q.om2[c]));
    for (int a = 0; a < P.n_orb; ++a)
        for (int c = 0; c < Q.n_orb; ++c) span = std::max(span, std::abs(P.om2[a] + Q.om2[c]));
    span += span & 1;                                  // keep 2m_a + 2m_b + span even
    if (2 * span + 1 > 255) return fail(CIH_ERR_UNSUPPORTED, "orbital 2m range too wide for the packed moves");
    X.m2span = span;
    X.G = (span + 1) * 2;
    X.S.assign((size_t)std::max(P.n_orb, 1) * X.G, 0);
    X.gsize.assign(X.G, 0);
    X.goff.assign(X.G, 0);
    X.rn.assign(std::max(Q.n_orb, 1), 0);
    for (int c = 0; c < Q.n_orb; ++c)
        for (int e = 0; e < c; ++e)
            if (Q.om2[e] == Q.om2[c] && ((Q.oN[e] ^ Q.oN[c]) & 1) == 0) X.rn[c]++;
    if (b.layout.total > INT32_MAX) return fail(CIH_ERR_UNSUPPORTED, "two-body table above 2^31 entries");
    std::vector<char> seen(X.S.size(), 0);
    for (int a = 0; a < P.n_orb; ++a)
        for (int c = 0; c < Q.n_orb; ++c) {
            int32_t code = b.layout.pid[(size_t)a * ntot + P.n_orb + c];
            if (code < 0) continue;
            int g = (code >> 16) & 0xFFF, u = code & 0xFFFF;
            int kappa = ((P.om2[a] + Q.om2[c] + span) / 2) * 2 + ((P.oN[a] + Q.oN[c]) & 1);
            int s = u - X.rn[c];
            size_t k = (size_t)a * X.G + kappa;
            if (seen[k] && X.S[k] != s) return fail(CIH_ERR_UNSUPPORTED, "internal: pn pair split inconsistent");
            if (s < INT16_MIN || s > INT16_MAX) return fail(CIH_ERR_UNSUPPORTED, "pn group too large");
            seen[k] = 1;
            X.S[k] = (int16_t)s;
            X.gsize[kappa] = b.layout.gsize[g];
            X.goff[kappa] = (int32_t)b.layout.goff[g];
        }
    return CIH_OK;
}

// One-body table layout: the combined orbitals stably sorted by (species, 2m,
// N parity); a run of equal keys is a group.
void build_onebody_layout(cih_basis &b)
{
    OneBodyLayout &L = b.onebody;
    const int np = b.s[0].n_orb, ntot = np + b.s[1].n_orb;
    auto key = [&](int a) {
        const Species &s = b.s[a < np ? 0 : 1];
        const int k = a < np ? a : a - np;
        return std::make_tuple(a < np ? 0 : 1, s.om2[k], s.oN[k] & 1);
    };
    std::vector<int> ord(ntot);
    for (int a = 0; a < ntot; ++a) ord[a] = a;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return key(x) < key(y); });
    L.grp.assign(std::max(ntot, 1), -1);
    L.loc.assign(std::max(ntot, 1), 0);
    L.gsize.clear();
    L.goff.clear();
    int64_t off = 0;
    for (int i = 0; i < ntot;) {
        int j = i;
        while (j < ntot && key(ord[j]) == key(ord[i])) ++j;
        const int g = (int)L.gsize.size(), n = j - i;
        for (int k = i; k < j; ++k) {
            L.grp[ord[k]] = (int16_t)g;
            L.loc[ord[k]] = (int16_t)(k - i);
        }
        L.gsize.push_back(n);
        L.goff.push_back((int32_t)off);
        off += (int64_t)n * (n + 1) / 2;
        i = j;
    }
    L.total = off;
}

}  // namespace

int build_host_species(const cih_space_t &sp, cih_basis &b)
{
    if (sp.Z < 0 || sp.N < 0 || sp.Nmax < 0) return fail(CIH_ERR_ARG, "Z, N and Nmax must be >= 0");
    if (sp.Z > 64 || sp.N > 64) return fail(CIH_ERR_UNSUPPORTED, "more than 64 particles of a species");
    b.space = sp;
    Timer tm("host basis");
    int Zs[2] = {sp.Z, sp.N};
    for (int t = 0; t < 2; ++t) {
        Species &s = b.s[t];
        s.Z = Zs[t];
        lowest_configuration(s.Z, s.N0, s.NF);
        if (s.Z > 0) {
            make_orbitals(s, s.NF + sp.Nmax);
        } else {
            s.oN.clear(); s.ol.clear(); s.oj2.clear(); s.om2.clear();
            s.n_orb = 0;
        }
        if (s.n_orb > 64 * kMaxWords) return fail(CIH_ERR_UNSUPPORTED, "more than 256 orbitals per species");
    }
    b.N0tot = b.s[0].N0 + b.s[1].N0;
    b.Nlim = b.N0tot + sp.Nmax;
    int words = 1;
    for (int t = 0; t < 2; ++t) {
        b.s[t].Nsub_max = b.Nlim - b.s[1 - t].N0;
        words = std::max(words, (b.s[t].n_orb + 63) / 64);
    }
    b.W = words <= 1 ? 1 : words <= 2 ? 2 : 4;

    // the two species are independent: count them side by side
    SubdetCount cnt[2];
    side_by_side([&]() { count_subdets(b.s[0], cnt[0]); }, [&]() { count_subdets(b.s[1], cnt[1]); });
    tm.mark("count p and n");

    // appearing buckets: those with a partner bucket of the other species
    std::vector<char> keep[2];
    for (int t = 0; t < 2; ++t) {
        const std::vector<std::pair<int, int>> mine = filled_buckets(b.s[t], cnt[t]);
        const std::vector<std::pair<int, int>> other = filled_buckets(b.s[1 - t], cnt[1 - t]);
        int mspan = std::abs(sp.twoM);
        for (const auto &q : other) mspan = std::max(mspan, std::abs(q.first));
        for (const auto &q : mine) mspan = std::max(mspan, std::abs(q.first) + std::abs(sp.twoM));
        std::vector<int> minN((size_t)(2 * mspan + 1) * 2, INT_MAX);   // (2M + mspan) * 2 + parity
        for (const auto &q : other) {
            int &m = minN[(size_t)(q.first + mspan) * 2 + (q.second & 1)];
            m = std::min(m, q.second);
        }
        if (b.s[t].Z == 0) {
            keep[t].assign(1, appears(0, 0, sp.twoM, b.Nlim, minN, mspan) ? 1 : 0);
        } else {
            keep[t].assign(cnt[t].nk, 0);
            for (int64_t k = 0; k < cnt[t].nk; ++k)
                keep[t][k] = cnt[t].total[k] > 0 &&
                             appears(cnt[t].M2_of(k), cnt[t].N_of(k), sp.twoM, b.Nlim, minN, mspan);
        }
    }
    side_by_side([&]() { write_subdets(b.s[0], cnt[0], keep[0]); },
                 [&]() { write_subdets(b.s[1], cnt[1], keep[1]); });
    tm.mark("appearing sub-dets written");
    side_by_side([&]() { make_classes(b.s[0]); }, [&]() { make_classes(b.s[1]); });
    tm.mark("appearing filter + classes");
    return CIH_OK;
}

int build_host_rest(cih_basis &b)
{
    Timer tm("host basis");
    const cih_space_t &sp = b.space;

    // partner ranges: class of (2M - 2M_p, parity of Nlim - N_p), prefix N <= Nlim - N_p
    const Species &P = b.s[0], &Q = b.s[1];
    int qspan = std::abs(sp.twoM);
    for (size_t c = 0; c < Q.cls_begin.size(); ++c) qspan = std::max(qspan, std::abs(Q.cls_M2[c]));
    for (int64_t i = 0; i < P.n_sd; ++i) qspan = std::max(qspan, std::abs(P.M2[i]) + std::abs(sp.twoM));
    std::vector<int> ncls((size_t)(2 * qspan + 1) * 2, -1);               // (2M + qspan) * 2 + parity
    for (size_t c = 0; c < Q.cls_begin.size(); ++c) ncls[(size_t)(Q.cls_M2[c] + qspan) * 2 + Q.cls_par[c]] = (int)c;
    std::vector<std::vector<int>> cum(Q.cls_begin.size());
    for (size_t c = 0; c < Q.cls_begin.size(); ++c) {
        cum[c].assign(b.Nlim + 2, 0);
        for (int i = Q.cls_begin[c]; i < Q.cls_end[c]; ++i) cum[c][Q.N[i] + 1]++;
        for (int L = 0; L <= b.Nlim; ++L) cum[c][L + 1] += cum[c][L];
    }
    b.nb.assign(P.n_sd, 0);
    b.nc.assign(P.n_sd, 0);
    b.rowbase.assign(P.n_sd + 1, 0);
    int64_t dim = 0;
    for (int64_t p = 0; p < P.n_sd; ++p) {
        int room = b.Nlim - P.N[p];
        const int mo = sp.twoM - P.M2[p];
        const int c = (room < 0 || mo < -qspan || mo > qspan) ? -1 : ncls[(size_t)(mo + qspan) * 2 + (room & 1)];
        if (c < 0) return fail(CIH_ERR_ARG, "internal: proton sub-det without partners");
        b.nb[p] = Q.cls_begin[c];
        b.nc[p] = cum[c][std::min(room, b.Nlim) + 1];
        b.rowbase[p] = dim;
        dim += b.nc[p];
    }
    b.rowbase[P.n_sd] = dim;
    b.dim = dim;
    if (dim > INT32_MAX) return fail(CIH_ERR_UNSUPPORTED, "dimension above 2^31-1 (int32 columns)");
    tm.mark("partner ranges");
    int rc = build_layout(b);
    tm.mark("table layout");
    if (rc) return rc;
    rc = build_pn_split(b);
    tm.mark("pn split");
    if (!rc) build_onebody_layout(b);
    return rc;
}

int build_host_basis(const cih_space_t &sp, cih_basis &b)
{
    int rc = build_host_species(sp, b);
    return rc ? rc : build_host_rest(b);
}

}  // namespace cih

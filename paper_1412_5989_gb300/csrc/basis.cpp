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
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <map>
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

struct Colex {
    const Species &s;
    std::vector<int> minsum;      // quanta of the c lowest orbitals
    uint64_t w[kMaxWords] = {0, 0, 0, 0};
    std::vector<uint64_t> bits;
    std::vector<int> N, M2;

    explicit Colex(const Species &sp) : s(sp)
    {
        minsum.assign(s.Z + 1, 0);
        for (int c = 1; c <= s.Z; ++c) minsum[c] = minsum[c - 1] + s.oN[c - 1];
    }

    // c more orbitals, all below `lim`, with at most `budget` quanta
    void rec(int c, int lim, int budget, int Nacc, int Macc)
    {
        if (c == 0) {
            bits.insert(bits.end(), w, w + kMaxWords);
            N.push_back(Nacc);
            M2.push_back(Macc);
            return;
        }
        for (int a = c - 1; a < lim; ++a) {
            if (s.oN[a] + minsum[c - 1] > budget) break;     // orbitals sorted by N
            w[a >> 6] |= 1ull << (a & 63);
            rec(c - 1, a, budget - s.oN[a], Nacc + s.oN[a], Macc + s.om2[a]);
            w[a >> 6] &= ~(1ull << (a & 63));
        }
    }
};

// stable counting sort of the generated sub-dets by (2M, N mod 2, N)
void bucket_sort(Species &s, Colex &g)
{
    int64_t n = (int64_t)g.N.size();
    int Mabs = 0;
    for (int m : g.M2) Mabs = std::max(Mabs, std::abs(m));
    int nN = s.Nsub_max + 1;
    auto key = [&](int64_t i) {
        return ((int64_t)(g.M2[i] + Mabs) * 2 + (g.N[i] & 1)) * nN + g.N[i];
    };
    int64_t nkeys = (int64_t)(2 * Mabs + 1) * 2 * nN;
    std::vector<int64_t> start(nkeys + 1, 0);
    for (int64_t i = 0; i < n; ++i) start[key(i) + 1]++;
    for (int64_t k = 0; k < nkeys; ++k) start[k + 1] += start[k];
    std::vector<int64_t> order(n);
    for (int64_t i = 0; i < n; ++i) order[start[key(i)]++] = i;
    s.n_sd = n;
    s.bits.resize((size_t)n * kMaxWords);
    s.N.resize(n);
    s.M2.resize(n);
    for (int64_t r = 0; r < n; ++r) {
        int64_t i = order[r];
        std::copy(&g.bits[i * kMaxWords], &g.bits[i * kMaxWords] + kMaxWords, &s.bits[r * kMaxWords]);
        s.N[r] = g.N[i];
        s.M2[r] = g.M2[i];
    }
}

void keep_only(Species &s, const std::vector<char> &keep)
{
    int64_t k = 0;
    for (int64_t i = 0; i < s.n_sd; ++i) {
        if (!keep[i]) continue;
        if (k != i) {
            std::copy(&s.bits[i * kMaxWords], &s.bits[i * kMaxWords] + kMaxWords, &s.bits[k * kMaxWords]);
            s.N[k] = s.N[i];
            s.M2[k] = s.M2[i];
        }
        ++k;
    }
    s.n_sd = k;
    s.bits.resize((size_t)k * kMaxWords);
    s.N.resize(k);
    s.M2.resize(k);
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
        std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> groups;
        for (int a = alo; a < ahi; ++a)
            for (int bb = std::max(blo, a + 1); bb < bhi; ++bb)
                if (orbN(a) + orbN(bb) <= limit)
                    groups[{orbM(a) + orbM(bb), (orbN(a) + orbN(bb)) & 1}].push_back({a, bb});
        int64_t off = 0;
        for (auto &kv : groups) {
            int g = (int)L.gsize.size();
            int n = (int)kv.second.size();
            if (g >= (1 << 12) || n >= (1 << 16)) return fail(CIH_ERR_UNSUPPORTED, "table group too large");
            L.gsize.push_back(n);
            L.goff.push_back(base + off);
            for (int u = 0; u < n; ++u) {
                int a = kv.second[u].first, bb = kv.second[u].second;
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

}  // namespace

int build_host_basis(const cih_space_t &sp, cih_basis &b)
{
    if (sp.Z < 0 || sp.N < 0 || sp.Nmax < 0) return fail(CIH_ERR_ARG, "Z, N and Nmax must be >= 0");
    if (sp.Z > 64 || sp.N > 64) return fail(CIH_ERR_UNSUPPORTED, "more than 64 particles of a species");
    b.space = sp;
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
        Species &s = b.s[t];
        s.Nsub_max = b.Nlim - b.s[1 - t].N0;
        Colex g(s);
        g.rec(s.Z, s.n_orb, s.Nsub_max, 0, 0);
        bucket_sort(s, g);
        words = std::max(words, (s.n_orb + 63) / 64);
    }
    b.W = words <= 1 ? 1 : words <= 2 ? 2 : 4;

    // appearing sub-dets: x pairs with some y of the other species when the
    // lowest-N partner of the right (2M, parity) fits under Nlim
    for (int t = 0; t < 2; ++t) {
        const Species &o = b.s[1 - t];
        std::map<std::pair<int, int>, int> minN;
        for (int64_t i = 0; i < o.n_sd; ++i) {
            auto k = std::make_pair(o.M2[i], o.N[i] & 1);
            auto it = minN.find(k);
            if (it == minN.end() || o.N[i] < it->second) minN[k] = o.N[i];
        }
        Species &s = b.s[t];
        std::vector<char> keep(s.n_sd, 0);
        for (int64_t i = 0; i < s.n_sd; ++i) {
            int room = b.Nlim - s.N[i];
            if (room < 0) continue;
            auto it = minN.find({sp.twoM - s.M2[i], room & 1});
            keep[i] = it != minN.end() && it->second <= room;
        }
        keep_only(s, keep);
    }
    // the filter of the second species used the first one's filtered list;
    // pairing is symmetric, so the first species' list is still exact.
    for (int t = 0; t < 2; ++t) make_classes(b.s[t]);

    // partner ranges: class of (2M - 2M_p, parity of Nlim - N_p), prefix N <= Nlim - N_p
    const Species &P = b.s[0], &Q = b.s[1];
    std::map<std::pair<int, int>, int> ncls;
    for (size_t c = 0; c < Q.cls_begin.size(); ++c) ncls[{Q.cls_M2[c], Q.cls_par[c]}] = (int)c;
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
        auto it = ncls.find({sp.twoM - P.M2[p], room & 1});
        if (room < 0 || it == ncls.end()) return fail(CIH_ERR_ARG, "internal: proton sub-det without partners");
        int c = it->second;
        b.nb[p] = Q.cls_begin[c];
        b.nc[p] = cum[c][std::min(room, b.Nlim) + 1];
        b.rowbase[p] = dim;
        dim += b.nc[p];
    }
    b.rowbase[P.n_sd] = dim;
    b.dim = dim;
    if (dim > INT32_MAX) return fail(CIH_ERR_UNSUPPORTED, "dimension above 2^31-1 (int32 columns)");
    int rc = build_layout(b);
    if (rc) return rc;
    return build_pn_split(b);
}

}  // namespace cih

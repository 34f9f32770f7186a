/*
 * cih_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU statement of what the library computes:
 * the M-scheme configuration-interaction Hamiltonian of the paper's Sec. 1-2
 * (the Schroedinger equation cast as a finite symmetric matrix eigenproblem over
 * a many-body basis, only half of the matrix stored), its lowest eigenpairs by
 * Lanczos (Sec. 2), and the derivative of the lowest eigenvalue with respect to
 * every two-body matrix element.
 *
 * Only tests, the smoke check and the timed CPU baseline of the benchmark may
 * load this library.  It shares no code, header, table or helper with the CUDA
 * library; the two meet only through seeded input tables that neither owns.
 *
 * Definitions (the paper states them in prose only; the readings are written
 * out in the design notes and repeated here where used):
 *   - single-particle orbitals per species: harmonic-oscillator (N,l,2j,2m)
 *     with N <= N_F + Nmax, ordered by (N,l,2j,2m) ascending;
 *   - Slater determinant |Phi> = a+_{i1} ... a+_{iA} |0>, i1 < ... < iA in the
 *     combined index (proton orbitals first, then neutron orbitals);
 *   - H = sum_a e_a a+_a a_a + sum_{a<b, c<d} V_{ab,cd} a+_a a+_b a_d a_c,
 *     e_a = hbar_omega (N_a + 3/2) unless a per-orbital table is given; or,
 *     with a one-body table t (or_set_onebody), H = sum_{a,c} t_ac a+_a a_c +
 *     the same two-body part, t symmetric and nonzero only between orbitals
 *     of one species with equal 2m and equal N parity (the paper's MFDn reads
 *     its one-body operator, the kinetic energy, from file: Sec. 2);
 *   - V_{ab,cd} is one real parameter that stands for both V_{ab,cd} and
 *     V_{cd,ab} (Hermiticity); a swapped pair changes its sign (antisymmetry).
 *
 * Nothing here is blocked, fused or reordered for speed beyond what these
 * definitions need; OpenMP only splits independent rows.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORW 8                 /* up to 512 orbitals per species */
#define ORCW (2 * ORW)        /* combined proton+neutron occupation words */

typedef struct { int N, l, j2, m2; } or_orb;

typedef struct {
    int npairs;
    int *pa, *pb;             /* combined orbital indices, pa < pb          */
    int ngroups;
    int *g_m2, *g_par, *g_first, *g_size;  /* group key, first pair, size  */
    long long *g_off;         /* offset of the group's packed triangle      */
    long long len;            /* entries in this channel                    */
    long long base;           /* offset of this channel in the whole table  */
} or_chan;

typedef struct {
    int Z[2], Nmax, twoM;
    int N0[2], NF[2], N0tot, Nlim;
    int norb[2];
    or_orb *orb[2];
    int ntot;                 /* n_orb_p + n_orb_n                           */
    long nsd[2];
    uint64_t *sd[2];          /* nsd x ORW words per species                 */
    int *sdN[2], *sdM[2];
    long *nbeg, *ncnt;        /* neutron partner range per proton sub-det    */
    long long *base;          /* first basis index of each proton sub-det    */
    long long dim;
    or_chan ch[3];            /* 0 = pp, 1 = nn, 2 = pn                      */
    long long tbme_len;
    int *pair_chan, *pair_grp, *pair_loc;   /* ntot x ntot lookup            */
    /* one-body layout: groups of orbitals of one species with equal (2m, N
       parity), in the order (species, 2m, parity) ascending, members ascending;
       each group stores its packed upper triangle (a <= c) */
    int ob_ngroups;
    int *ob_grp, *ob_loc;     /* per combined orbital: group, place in it      */
    int *ob_gsize, *ob_gfirst, *ob_orb;     /* group size, first member, members */
    long long *ob_goff;       /* offset of each group's triangle              */
    long long ob_len;
    const double *t1;         /* the one-body table in use, or NULL           */
} or_space;

/* ------------------------------------------------------------------ */
/* single-particle basis                                              */
/* ------------------------------------------------------------------ */

/* minimal total oscillator quanta of k particles of one species, and the
   highest shell they touch: fill shells of capacity (N+1)(N+2) from N = 0 */
static void lowest_config(int k, int *N0, int *NF)
{
    int left = k, N = 0, sum = 0, top = -1;
    while (left > 0) {
        int cap = (N + 1) * (N + 2);
        int put = left < cap ? left : cap;
        sum += put * N;
        left -= put;
        top = N;
        N++;
    }
    *N0 = sum;
    *NF = top;
}

static int make_orbitals(int Nshell_max, or_orb *out)
{
    int k = 0;
    for (int N = 0; N <= Nshell_max; N++)
        for (int l = N % 2; l <= N; l += 2)
            for (int j2 = 2 * l - 1; j2 <= 2 * l + 1; j2 += 2) {
                if (j2 < 0) continue;
                for (int m2 = -j2; m2 <= j2; m2 += 2) {
                    if (out) { out[k].N = N; out[k].l = l; out[k].j2 = j2; out[k].m2 = m2; }
                    k++;
                }
            }
    return k;
}

/* ------------------------------------------------------------------ */
/* sub-determinants                                                   */
/* ------------------------------------------------------------------ */

typedef struct { uint64_t w[ORW]; int N, M; } sdtmp;

typedef struct { sdtmp *v; long n, cap; } sdlist;

static void push(sdlist *L, const uint64_t *w, int N, int M)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 256;
        L->v = (sdtmp *)realloc(L->v, (size_t)L->cap * sizeof(sdtmp));
    }
    memcpy(L->v[L->n].w, w, sizeof(uint64_t) * ORW);
    L->v[L->n].N = N;
    L->v[L->n].M = M;
    L->n++;
}

/* every k-subset of the orbitals whose quanta sum stays <= Nsub_max */
static void subsets(const or_orb *orb, int norb, int first, int k, int Nacc,
                    int Nsub_max, int Macc, uint64_t *w, sdlist *L)
{
    if (k == 0) { push(L, w, Nacc, Macc); return; }
    for (int a = first; a < norb; a++) {
        if (Nacc + orb[a].N > Nsub_max) continue;
        w[a >> 6] |= 1ull << (a & 63);
        subsets(orb, norb, a + 1, k - 1, Nacc + orb[a].N, Nsub_max, Macc + orb[a].m2, w, L);
        w[a >> 6] &= ~(1ull << (a & 63));
    }
}

/* order key (2M, N mod 2, N, bit string as an unsigned multiword integer) */
static int sd_cmp(const void *x, const void *y)
{
    const sdtmp *a = (const sdtmp *)x, *b = (const sdtmp *)y;
    if (a->M != b->M) return a->M < b->M ? -1 : 1;
    if ((a->N & 1) != (b->N & 1)) return (a->N & 1) < (b->N & 1) ? -1 : 1;
    if (a->N != b->N) return a->N < b->N ? -1 : 1;
    for (int w = ORW - 1; w >= 0; w--)
        if (a->w[w] != b->w[w]) return a->w[w] < b->w[w] ? -1 : 1;
    return 0;
}

static int popc_words(const uint64_t *a, int n)
{
    int c = 0;
    for (int i = 0; i < n; i++) c += __builtin_popcountll(a[i]);
    return c;
}

/* ------------------------------------------------------------------ */
/* the many-body basis                                                */
/* ------------------------------------------------------------------ */

static void free_chan(or_chan *c)
{
    free(c->pa); free(c->pb); free(c->g_m2); free(c->g_par);
    free(c->g_first); free(c->g_size); free(c->g_off);
}

void or_space_free(or_space *S)
{
    if (!S) return;
    for (int s = 0; s < 2; s++) {
        free(S->orb[s]); free(S->sd[s]); free(S->sdN[s]); free(S->sdM[s]);
    }
    free(S->nbeg); free(S->ncnt); free(S->base);
    for (int c = 0; c < 3; c++) free_chan(&S->ch[c]);
    free(S->pair_chan); free(S->pair_grp); free(S->pair_loc);
    free(S->ob_grp); free(S->ob_loc); free(S->ob_gsize); free(S->ob_gfirst); free(S->ob_orb); free(S->ob_goff);
    free(S);
}

static int orb_N(const or_space *S, int a)
{
    return a < S->norb[0] ? S->orb[0][a].N : S->orb[1][a - S->norb[0]].N;
}
static int orb_m2(const or_space *S, int a)
{
    return a < S->norb[0] ? S->orb[0][a].m2 : S->orb[1][a - S->norb[0]].m2;
}

/* Two-body table layout (the input format): channels pp, nn, pn; a pair
   (a<b) belongs to its channel when N_a + N_b <= Nlim - N0(other A-2
   particles); pairs are grouped by (2M_pair, parity) ascending and ordered
   (a,b) lexicographically inside a group; a group stores its packed
   row-major upper triangle (bra pair <= ket pair). */
static void build_channel(or_space *S, int c)
{
    or_chan *C = &S->ch[c];
    memset(C, 0, sizeof(*C));
    int zp = S->Z[0], zn = S->Z[1];
    int need_p = (c == 0) ? 2 : (c == 1) ? 0 : 1;
    int need_n = (c == 0) ? 0 : (c == 1) ? 2 : 1;
    if (zp < need_p || zn < need_n) return;
    int n0p, n0n, dummy;
    lowest_config(zp - need_p, &n0p, &dummy);
    lowest_config(zn - need_n, &n0n, &dummy);
    int Npair_max = S->Nlim - (n0p + n0n);

    int lo_a = (c == 1) ? S->norb[0] : 0;
    int hi_a = (c == 0) ? S->norb[0] : (c == 1) ? S->ntot : S->norb[0];
    int lo_b = (c == 0) ? 0 : S->norb[0];
    int hi_b = (c == 0) ? S->norb[0] : S->ntot;

    /* collect pairs with their group keys, then stable sort by group */
    int cap = 1024, n = 0;
    int *pa = (int *)malloc(sizeof(int) * cap), *pb = (int *)malloc(sizeof(int) * cap);
    for (int a = lo_a; a < hi_a; a++)
        for (int b = (lo_b > a + 1 ? lo_b : a + 1); b < hi_b; b++) {
            if (orb_N(S, a) + orb_N(S, b) > Npair_max) continue;
            if (n == cap) {
                cap *= 2;
                pa = (int *)realloc(pa, sizeof(int) * cap);
                pb = (int *)realloc(pb, sizeof(int) * cap);
            }
            pa[n] = a; pb[n] = b; n++;
        }
    /* distinct group keys, ascending */
    int gcap = 64, ng = 0;
    int *gm = (int *)malloc(sizeof(int) * gcap), *gp = (int *)malloc(sizeof(int) * gcap);
    for (int i = 0; i < n; i++) {
        int m = orb_m2(S, pa[i]) + orb_m2(S, pb[i]);
        int p = (orb_N(S, pa[i]) + orb_N(S, pb[i])) & 1;
        int found = 0;
        for (int g = 0; g < ng; g++) if (gm[g] == m && gp[g] == p) { found = 1; break; }
        if (!found) {
            if (ng == gcap) { gcap *= 2; gm = (int *)realloc(gm, sizeof(int) * gcap); gp = (int *)realloc(gp, sizeof(int) * gcap); }
            gm[ng] = m; gp[ng] = p; ng++;
        }
    }
    /* insertion sort of the (few) group keys */
    for (int i = 1; i < ng; i++)
        for (int j = i; j > 0 && (gm[j - 1] > gm[j] || (gm[j - 1] == gm[j] && gp[j - 1] > gp[j])); j--) {
            int t = gm[j]; gm[j] = gm[j - 1]; gm[j - 1] = t;
            t = gp[j]; gp[j] = gp[j - 1]; gp[j - 1] = t;
        }
    C->npairs = n;
    C->pa = (int *)malloc(sizeof(int) * (n ? n : 1));
    C->pb = (int *)malloc(sizeof(int) * (n ? n : 1));
    C->ngroups = ng;
    C->g_m2 = gm; C->g_par = gp;
    C->g_first = (int *)malloc(sizeof(int) * (ng ? ng : 1));
    C->g_size = (int *)malloc(sizeof(int) * (ng ? ng : 1));
    C->g_off = (long long *)malloc(sizeof(long long) * (ng ? ng : 1));
    int k = 0;
    long long off = 0;
    for (int g = 0; g < ng; g++) {
        C->g_first[g] = k;
        for (int i = 0; i < n; i++) {   /* pairs were generated in lexicographic order */
            int m = orb_m2(S, pa[i]) + orb_m2(S, pb[i]);
            int p = (orb_N(S, pa[i]) + orb_N(S, pb[i])) & 1;
            if (m == gm[g] && p == gp[g]) { C->pa[k] = pa[i]; C->pb[k] = pb[i]; k++; }
        }
        C->g_size[g] = k - C->g_first[g];
        C->g_off[g] = off;
        off += (long long)C->g_size[g] * (C->g_size[g] + 1) / 2;
    }
    C->len = off;
    free(pa); free(pb);
}

/* One-body table layout (see or_space).  Plain quadratic scans over the
   orbitals: a group is every orbital of species s with the key (2m, parity). */
static void build_onebody_layout(or_space *S)
{
    int nt = S->ntot > 0 ? S->ntot : 1;
    S->ob_grp = (int *)malloc(sizeof(int) * nt);
    S->ob_loc = (int *)malloc(sizeof(int) * nt);
    S->ob_orb = (int *)malloc(sizeof(int) * nt);
    S->ob_gsize = (int *)malloc(sizeof(int) * nt);
    S->ob_gfirst = (int *)malloc(sizeof(int) * nt);
    S->ob_goff = (long long *)malloc(sizeof(long long) * nt);
    for (int a = 0; a < S->ntot; a++) S->ob_grp[a] = -1;
    int g = 0, placed = 0;
    long long off = 0;
    for (int s = 0; s < 2; s++) {
        int base = s ? S->norb[0] : 0;
        for (int m2 = -4 * ORW * 64; m2 <= 4 * ORW * 64; m2++)        /* 2m ascending */
            for (int par = 0; par < 2; par++) {
                int n = 0;
                for (int a = 0; a < S->norb[s]; a++) {
                    const or_orb *o = &S->orb[s][a];
                    if (o->m2 != m2 || (o->N & 1) != par) continue;
                    S->ob_grp[base + a] = g;
                    S->ob_loc[base + a] = n;
                    S->ob_orb[placed + n] = base + a;
                    n++;
                }
                if (!n) continue;
                S->ob_gsize[g] = n;
                S->ob_gfirst[g] = placed;
                S->ob_goff[g] = off;
                off += (long long)n * (n + 1) / 2;
                placed += n;
                g++;
            }
    }
    S->ob_ngroups = g;
    S->ob_len = off;
}

/* table index of t_ac (either order), or -1 if a and c are not in one group */
long long or_onebody_index(const or_space *S, int a, int c)
{
    if (a < 0 || c < 0 || a >= S->ntot || c >= S->ntot) return -1;
    int g = S->ob_grp[a];
    if (g < 0 || g != S->ob_grp[c]) return -1;
    long long u = S->ob_loc[a], v = S->ob_loc[c];
    if (u > v) { long long t = u; u = v; v = t; }
    long long n = S->ob_gsize[g];
    return S->ob_goff[g] + u * n - u * (u - 1) / 2 + (v - u);
}

long long or_onebody_len(const or_space *S) { return S->ob_len; }

/* use t (ob_len doubles, kept alive by the caller) as the one-body part of H
   for later element, dense and row calls; NULL returns to e_a / hbar_omega */
void or_set_onebody(or_space *S, const double *t1) { S->t1 = t1; }

or_space *or_space_new(int Zp, int Zn, int Nmax, int twoM)
{
    if (Zp < 0 || Zn < 0 || Nmax < 0) return NULL;
    or_space *S = (or_space *)calloc(1, sizeof(or_space));
    S->Z[0] = Zp; S->Z[1] = Zn; S->Nmax = Nmax; S->twoM = twoM;
    for (int s = 0; s < 2; s++) lowest_config(S->Z[s], &S->N0[s], &S->NF[s]);
    S->N0tot = S->N0[0] + S->N0[1];
    S->Nlim = S->N0tot + Nmax;
    for (int s = 0; s < 2; s++) {
        if (S->Z[s] == 0) { S->norb[s] = 0; S->orb[s] = (or_orb *)malloc(sizeof(or_orb)); continue; }
        int n = make_orbitals(S->NF[s] + Nmax, NULL);
        if (n > 64 * ORW) { or_space_free(S); return NULL; }
        S->norb[s] = n;
        S->orb[s] = (or_orb *)malloc(sizeof(or_orb) * n);
        make_orbitals(S->NF[s] + Nmax, S->orb[s]);
    }
    S->ntot = S->norb[0] + S->norb[1];

    /* all truncated sub-determinants of each species */
    sdlist L[2] = {{0}, {0}};
    for (int s = 0; s < 2; s++) {
        uint64_t w[ORW] = {0};
        subsets(S->orb[s], S->norb[s], 0, S->Z[s], 0, S->N0[s] + Nmax, 0, w, &L[s]);
    }
    /* keep the ones that appear in at least one basis state: x appears when
       the other species has some sub-determinant with 2M = twoM - 2M_x and an
       N of the right parity that keeps N_tot <= Nlim */
    int Mspan = 0;
    for (int s = 0; s < 2; s++)
        for (long i = 0; i < L[s].n; i++)
            if (abs(L[s].v[i].M) > Mspan) Mspan = abs(L[s].v[i].M);
    int nM = 2 * Mspan + 1, nN = S->Nlim + 1;
    char *has[2];
    for (int s = 0; s < 2; s++) {
        has[s] = (char *)calloc((size_t)nM * nN, 1);
        for (long i = 0; i < L[s].n; i++)
            if (L[s].v[i].N <= S->Nlim) has[s][(size_t)(L[s].v[i].M + Mspan) * nN + L[s].v[i].N] = 1;
    }
    long kept[2];
    for (int s = 0; s < 2; s++) {
        long keep = 0;
        for (long i = 0; i < L[s].n; i++) {
            int Mo = twoM - L[s].v[i].M, ok = 0;
            if (Mo >= -Mspan && Mo <= Mspan)
                for (int No = 0; No + L[s].v[i].N <= S->Nlim; No++)
                    if (((No + L[s].v[i].N - S->Nlim) % 2 == 0) && has[1 - s][(size_t)(Mo + Mspan) * nN + No]) ok = 1;
            if (ok) L[s].v[keep++] = L[s].v[i];
        }
        kept[s] = keep;
    }
    for (int s = 0; s < 2; s++) { L[s].n = kept[s]; free(has[s]); }
    for (int s = 0; s < 2; s++) {
        qsort(L[s].v, (size_t)L[s].n, sizeof(sdtmp), sd_cmp);
        S->nsd[s] = L[s].n;
        long n = L[s].n ? L[s].n : 1;
        S->sd[s] = (uint64_t *)calloc((size_t)n * ORW, sizeof(uint64_t));
        S->sdN[s] = (int *)malloc(sizeof(int) * n);
        S->sdM[s] = (int *)malloc(sizeof(int) * n);
        for (long i = 0; i < L[s].n; i++) {
            memcpy(&S->sd[s][i * ORW], L[s].v[i].w, sizeof(uint64_t) * ORW);
            S->sdN[s][i] = L[s].v[i].N;
            S->sdM[s][i] = L[s].v[i].M;
        }
        free(L[s].v);
    }
    /* basis: (p, n) pairs in lexicographic order */
    long np = S->nsd[0], nn = S->nsd[1];
    S->nbeg = (long *)malloc(sizeof(long) * (np ? np : 1));
    S->ncnt = (long *)malloc(sizeof(long) * (np ? np : 1));
    S->base = (long long *)malloc(sizeof(long long) * (np + 1));
    long long dim = 0;
    for (long p = 0; p < np; p++) {
        /* partners: 2M_n = twoM - 2M_p, N_n of parity (Nlim - N_p), N_n <= Nlim - N_p;
           in the (2M, N mod 2, N, bits) order they start at the first sub-det of
           that (2M, parity) class and run while N_n stays under the limit */
        int Mn = twoM - S->sdM[0][p], Ln = S->Nlim - S->sdN[0][p], par = ((Ln % 2) + 2) % 2;
        long lo = 0, hi = nn;
        while (lo < hi) {
            long mid = (lo + hi) / 2;
            int mM = S->sdM[1][mid], mP = S->sdN[1][mid] & 1;
            if (mM < Mn || (mM == Mn && mP < par)) lo = mid + 1; else hi = mid;
        }
        long cnt = 0;
        while (lo + cnt < nn && S->sdM[1][lo + cnt] == Mn && (S->sdN[1][lo + cnt] & 1) == par &&
               S->sdN[1][lo + cnt] <= Ln)
            cnt++;
        S->nbeg[p] = lo;
        S->ncnt[p] = cnt;
        S->base[p] = dim;
        dim += cnt;
    }
    S->base[np] = dim;
    S->dim = dim;

    /* two-body table layout */
    S->pair_chan = (int *)malloc(sizeof(int) * (size_t)(S->ntot ? S->ntot * S->ntot : 1));
    S->pair_grp = (int *)malloc(sizeof(int) * (size_t)(S->ntot ? S->ntot * S->ntot : 1));
    S->pair_loc = (int *)malloc(sizeof(int) * (size_t)(S->ntot ? S->ntot * S->ntot : 1));
    for (long i = 0; i < (long)S->ntot * S->ntot; i++) S->pair_chan[i] = -1;
    long long tot = 0;
    for (int c = 0; c < 3; c++) {
        build_channel(S, c);
        S->ch[c].base = tot;
        tot += S->ch[c].len;
        for (int g = 0; g < S->ch[c].ngroups; g++)
            for (int u = 0; u < S->ch[c].g_size[g]; u++) {
                int k = S->ch[c].g_first[g] + u;
                long idx = (long)S->ch[c].pa[k] * S->ntot + S->ch[c].pb[k];
                S->pair_chan[idx] = c;
                S->pair_grp[idx] = g;
                S->pair_loc[idx] = u;
            }
    }
    S->tbme_len = tot;
    build_onebody_layout(S);
    return S;
}

/* ------------------------------------------------------------------ */
/* queries                                                            */
/* ------------------------------------------------------------------ */

void or_space_info(const or_space *S, long long *dim, int *norb, long *nsd,
                   long long *chan_len, long long *tbme_len)
{
    *dim = S->dim;
    norb[0] = S->norb[0]; norb[1] = S->norb[1];
    nsd[0] = S->nsd[0]; nsd[1] = S->nsd[1];
    for (int c = 0; c < 3; c++) chan_len[c] = S->ch[c].len;
    *tbme_len = S->tbme_len;
}

void or_orbitals(const or_space *S, int s, int *out4)
{
    for (int a = 0; a < S->norb[s]; a++) {
        out4[4 * a] = S->orb[s][a].N; out4[4 * a + 1] = S->orb[s][a].l;
        out4[4 * a + 2] = S->orb[s][a].j2; out4[4 * a + 3] = S->orb[s][a].m2;
    }
}

/* sub-determinant bit strings, ORW words each, and (N, 2M) */
void or_subdets(const or_space *S, int s, uint64_t *words, int *N, int *M)
{
    memcpy(words, S->sd[s], sizeof(uint64_t) * ORW * (size_t)S->nsd[s]);
    memcpy(N, S->sdN[s], sizeof(int) * (size_t)S->nsd[s]);
    memcpy(M, S->sdM[s], sizeof(int) * (size_t)S->nsd[s]);
}

void or_partner_ranges(const or_space *S, long *nbeg, long *ncnt, long long *base)
{
    for (long p = 0; p < S->nsd[0]; p++) { nbeg[p] = S->nbeg[p]; ncnt[p] = S->ncnt[p]; base[p] = S->base[p]; }
    base[S->nsd[0]] = S->dim;
}

/* pair list of one channel: combined indices and group of each pair */
long or_channel_pairs(const or_space *S, int c, int *pa, int *pb, int *grp)
{
    const or_chan *C = &S->ch[c];
    if (pa) {
        for (int g = 0; g < C->ngroups; g++)
            for (int u = 0; u < C->g_size[g]; u++) {
                int k = C->g_first[g] + u;
                pa[k] = C->pa[k]; pb[k] = C->pb[k]; grp[k] = g;
            }
    }
    return C->npairs;
}

static void basis_split(const or_space *S, long long i, long *p, long *n)
{
    long lo = 0, hi = S->nsd[0] - 1;
    while (lo < hi) {                 /* last p with base[p] <= i and ncnt > 0 */
        long mid = (lo + hi + 1) / 2;
        if (S->base[mid] <= i) lo = mid; else hi = mid - 1;
    }
    while (S->ncnt[lo] == 0) lo--;    /* cannot happen: every kept p has partners */
    *p = lo;
    *n = S->nbeg[lo] + (long)(i - S->base[lo]);
}

/* combined occupation bits of basis state i: ORCW words, proton orbital a at
   bit a, neutron orbital b at bit n_orb_p + b */
static void state_occ(const or_space *S, long long i, uint64_t *occ)
{
    long p, n;
    basis_split(S, i, &p, &n);
    memset(occ, 0, sizeof(uint64_t) * ORCW);
    for (int a = 0; a < S->norb[0]; a++)
        if (S->sd[0][p * ORW + (a >> 6)] >> (a & 63) & 1) occ[a >> 6] |= 1ull << (a & 63);
    for (int b = 0; b < S->norb[1]; b++)
        if (S->sd[1][n * ORW + (b >> 6)] >> (b & 63) & 1) {
            int k = S->norb[0] + b;
            occ[k >> 6] |= 1ull << (k & 63);
        }
}

void or_basis_state(const or_space *S, long long i, long *p, long *n) { basis_split(S, i, p, n); }

static int occ_bit(const uint64_t *o, int k) { return (int)(o[k >> 6] >> (k & 63) & 1); }

/* number of occupied orbitals with index < k */
static int occ_below(const uint64_t *o, int k)
{
    int c = 0;
    for (int w = 0; w < (k >> 6); w++) c += __builtin_popcountll(o[w]);
    if (k & 63) c += __builtin_popcountll(o[k >> 6] & ((1ull << (k & 63)) - 1));
    return c;
}

/* a_k: returns 0 if empty, else the sign (-1)^(occupied below k) */
static int annihilate(uint64_t *o, int k)
{
    if (!occ_bit(o, k)) return 0;
    int s = (occ_below(o, k) & 1) ? -1 : 1;
    o[k >> 6] &= ~(1ull << (k & 63));
    return s;
}
static int create(uint64_t *o, int k)
{
    if (occ_bit(o, k)) return 0;
    int s = (occ_below(o, k) & 1) ? -1 : 1;
    o[k >> 6] |= 1ull << (k & 63);
    return s;
}

/* basis index of a combined occupation, or -1 if it is not a basis state */
static long long occ_index(const or_space *S, const uint64_t *occ)
{
    uint64_t w[2][ORW];
    memset(w, 0, sizeof(w));
    int Nsub[2] = {0, 0}, Msub[2] = {0, 0}, cnt[2] = {0, 0};
    for (int k = 0; k < S->ntot; k++) {
        if (!occ_bit(occ, k)) continue;
        int s = k < S->norb[0] ? 0 : 1;
        int a = s ? k - S->norb[0] : k;
        w[s][a >> 6] |= 1ull << (a & 63);
        Nsub[s] += S->orb[s][a].N;
        Msub[s] += S->orb[s][a].m2;
        cnt[s]++;
    }
    if (cnt[0] != S->Z[0] || cnt[1] != S->Z[1]) return -1;
    long idx[2];
    for (int s = 0; s < 2; s++) {
        sdtmp key;
        memcpy(key.w, w[s], sizeof(key.w));
        key.N = Nsub[s]; key.M = Msub[s];
        long lo = 0, hi = S->nsd[s];
        while (lo < hi) {
            long mid = (lo + hi) / 2;
            sdtmp m;
            memcpy(m.w, &S->sd[s][mid * ORW], sizeof(m.w));
            m.N = S->sdN[s][mid]; m.M = S->sdM[s][mid];
            if (sd_cmp(&m, &key) < 0) lo = mid + 1; else hi = mid;
        }
        if (lo >= S->nsd[s]) return -1;
        if (memcmp(&S->sd[s][lo * ORW], w[s], sizeof(uint64_t) * ORW) != 0) return -1;
        idx[s] = lo;
    }
    long p = idx[0], n = idx[1];
    if (n < S->nbeg[p] || n >= S->nbeg[p] + S->ncnt[p]) return -1;
    return S->base[p] + (n - S->nbeg[p]);
}

/* ------------------------------------------------------------------ */
/* two-body matrix elements                                           */
/* ------------------------------------------------------------------ */

/* table index and sign of V_{ab,cd} for any orbital order; -1 if the element
   is not a table entry (different channel or group, or outside the layout) */
long long or_tbme_index(const or_space *S, int a, int b, int c, int d, int *sign)
{
    int s = 1;
    *sign = 0;
    if (a == b || c == d) return -1;
    if (a > b) { int t = a; a = b; b = t; s = -s; }
    if (c > d) { int t = c; c = d; d = t; s = -s; }
    long i1 = (long)a * S->ntot + b, i2 = (long)c * S->ntot + d;
    int c1 = S->pair_chan[i1], c2 = S->pair_chan[i2];
    if (c1 < 0 || c1 != c2) return -1;
    if (S->pair_grp[i1] != S->pair_grp[i2]) return -1;
    const or_chan *C = &S->ch[c1];
    int g = S->pair_grp[i1];
    long long u = S->pair_loc[i1], v = S->pair_loc[i2];
    if (u > v) { long long t = u; u = v; v = t; }
    long long n = C->g_size[g];
    *sign = s;
    return C->base + C->g_off[g] + u * n - u * (u - 1) / 2 + (v - u);
}

static double one_body(const or_space *S, const double *esp, double hw, int a)
{
    if (S->t1) return S->t1[or_onebody_index(S, a, a)];
    if (esp) return esp[a];
    return hw * (orb_N(S, a) + 1.5);
}

static int vlookup(const or_space *S, const float *tbme, int a, int b, int c, int d, double *v)
{
    int sg;
    long long idx = or_tbme_index(S, a, b, c, d, &sg);
    if (idx < 0) return -1;
    *v = sg * (double)tbme[idx];
    return 0;
}

/* <Phi_i | H | Phi_j> by the Slater-Condon reduction of the definition:
   the ket and bra differ in 0, 1 or 2 orbitals, and each case keeps only the
   operator terms that connect them.  FP64 sum in a fixed order (one-body
   terms by orbital, then two-body terms by ascending spectator / pair).
   Returns 1 if (i,j) is structurally connected (<= 2 particles moved). */
int or_element(const or_space *S, const float *tbme, const double *esp, double hw,
               long long i, long long j, double *out)
{
    uint64_t oi[ORCW], oj[ORCW], x[ORCW];
    state_occ(S, i, oi);
    state_occ(S, j, oj);
    int nd = 0;
    for (int w = 0; w < ORCW; w++) { x[w] = oi[w] ^ oj[w]; nd += __builtin_popcountll(x[w]); }
    nd /= 2;
    *out = 0.0;
    if (nd > 2) return 0;
    double sum = 0.0, v;
    if (nd == 0) {
        for (int a = 0; a < S->ntot; a++) if (occ_bit(oj, a)) sum += one_body(S, esp, hw, a);
        for (int a = 0; a < S->ntot; a++) {
            if (!occ_bit(oj, a)) continue;
            for (int b = a + 1; b < S->ntot; b++) {
                if (!occ_bit(oj, b)) continue;
                if (vlookup(S, tbme, a, b, a, b, &v)) return -1;
                sum += v;
            }
        }
        *out = sum;
        return 1;
    }
    int in_i[2] = {0, 0}, in_j[2] = {0, 0}, ni = 0, nj = 0;   /* ascending */
    for (int k = 0; k < S->ntot; k++) {
        if (occ_bit(x, k) && occ_bit(oi, k)) in_i[ni++] = k;
        if (occ_bit(x, k) && occ_bit(oj, k)) in_j[nj++] = k;
    }
    if (nd == 1) {
        int a = in_i[0], c = in_j[0];
        uint64_t t[ORCW];
        memcpy(t, oj, sizeof(t));
        int s = annihilate(t, c);
        s *= create(t, a);                    /* a+_a a_c |Phi_j> = s |Phi_i> */
        if (S->t1) {                          /* the one-body term first */
            long long k1 = or_onebody_index(S, a, c);
            if (k1 < 0) return -1;
            sum += S->t1[k1];
        }
        for (int k = 0; k < S->ntot; k++) {
            if (!occ_bit(oj, k) || k == c) continue;     /* spectators, ascending */
            if (vlookup(S, tbme, a, k, c, k, &v)) return -1;
            sum += v;
        }
        *out = s * sum;
        return 1;
    }
    /* nd == 2: a<b created, c<d annihilated */
    int a = in_i[0], b = in_i[1], c = in_j[0], d = in_j[1];
    uint64_t t[ORCW];
    memcpy(t, oj, sizeof(t));
    int s = annihilate(t, c);
    s *= annihilate(t, d);
    s *= create(t, b);
    s *= create(t, a);                        /* a+_a a+_b a_d a_c |Phi_j> */
    if (vlookup(S, tbme, a, b, c, d, &v)) return -1;   /* every needed pair is in the layout */
    *out = s * v;
    return 1;
}

/* Dense H (row-major dim x dim, FP64) by applying every operator term of the
   definition to every ket with explicit sign counting ("brute force"):
   H|Phi_j> = sum_terms coefficient * (operator |Phi_j>), and each image that is
   a basis state |Phi_i> adds to H[i][j].  Tiny bases only. */
int or_dense_brute(const or_space *S, const float *tbme, const double *esp, double hw, double *H)
{
    long long D = S->dim;
    memset(H, 0, sizeof(double) * (size_t)(D * D));
    uint64_t o[ORCW], t[ORCW];
    for (long long j = 0; j < D; j++) {
        state_occ(S, j, o);
        for (int a = 0; a < S->ntot; a++)
            if (occ_bit(o, a)) H[j * D + j] += one_body(S, esp, hw, a);
        if (S->t1)                            /* t_ac a+_a a_c, a != c, both orders */
            for (int g = 0; g < S->ob_ngroups; g++) {
                int n = S->ob_gsize[g];
                for (int u = 0; u < n; u++)
                    for (int w = 0; w < n; w++) {
                        if (u == w) continue;
                        int a = S->ob_orb[S->ob_gfirst[g] + u], c = S->ob_orb[S->ob_gfirst[g] + w];
                        memcpy(t, o, sizeof(t));
                        int s = annihilate(t, c);
                        if (!s) continue;
                        s *= create(t, a);
                        if (!s) continue;
                        long long i = occ_index(S, t);
                        if (i < 0) continue;
                        H[i * D + j] += s * S->t1[or_onebody_index(S, a, c)];
                    }
            }
        for (int c3 = 0; c3 < 3; c3++) {
            const or_chan *C = &S->ch[c3];
            for (int g = 0; g < C->ngroups; g++) {
                int n = C->g_size[g];
                for (int u = 0; u < n; u++)
                    for (int w = u; w < n; w++) {
                        long long idx = C->base + C->g_off[g] + (long long)u * n - (long long)u * (u - 1) / 2 + (w - u);
                        double val = tbme[idx];
                        for (int herm = 0; herm < (u == w ? 1 : 2); herm++) {
                            int bra = herm ? C->g_first[g] + w : C->g_first[g] + u;
                            int ket = herm ? C->g_first[g] + u : C->g_first[g] + w;
                            int pa = C->pa[bra], pb = C->pb[bra], pc = C->pa[ket], pd = C->pb[ket];
                            memcpy(t, o, sizeof(t));
                            int s = annihilate(t, pc);
                            if (!s) continue;
                            s *= annihilate(t, pd);
                            if (!s) continue;
                            s *= create(t, pb);
                            if (!s) continue;
                            s *= create(t, pa);
                            if (!s) continue;
                            long long i = occ_index(S, t);
                            if (i < 0) continue;
                            H[i * D + j] += s * val;
                        }
                    }
            }
        }
    }
    return 0;
}

/* d H / d t for one table parameter t, applied ket-driven as above, folded
   into <psi| dH/dt |psi> (the two-body density of the parameter's operator
   plus its Hermitian partner).  Tiny bases only. */
void or_density_brute(const or_space *S, const double *psi, double *grad)
{
    long long D = S->dim;
    memset(grad, 0, sizeof(double) * (size_t)S->tbme_len);
    uint64_t o[ORCW], t[ORCW];
    for (long long j = 0; j < D; j++) {
        if (psi[j] == 0.0) continue;
        state_occ(S, j, o);
        for (int c3 = 0; c3 < 3; c3++) {
            const or_chan *C = &S->ch[c3];
            for (int g = 0; g < C->ngroups; g++) {
                int n = C->g_size[g];
                for (int u = 0; u < n; u++)
                    for (int w = u; w < n; w++) {
                        long long idx = C->base + C->g_off[g] + (long long)u * n - (long long)u * (u - 1) / 2 + (w - u);
                        for (int herm = 0; herm < (u == w ? 1 : 2); herm++) {
                            int bra = herm ? C->g_first[g] + w : C->g_first[g] + u;
                            int ket = herm ? C->g_first[g] + u : C->g_first[g] + w;
                            memcpy(t, o, sizeof(t));
                            int s = annihilate(t, C->pa[ket]);
                            if (!s) continue;
                            s *= annihilate(t, C->pb[ket]);
                            if (!s) continue;
                            s *= create(t, C->pb[bra]);
                            if (!s) continue;
                            s *= create(t, C->pa[bra]);
                            if (!s) continue;
                            long long i = occ_index(S, t);
                            if (i < 0) continue;
                            grad[idx] += s * psi[i] * psi[j];
                        }
                    }
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* half-stored CSR by the plain row walk                              */
/* ------------------------------------------------------------------ */

/* A column j >= i is stored when its determinant differs from row i's by at
   most two particles (popcount of the XOR <= 4), whatever the value.  The walk
   visits proton sub-determinants in order and, for each within two moves, the
   neutron partners of its range: the columns come out ascending. */
static long row_walk(const or_space *S, const float *tbme, const double *esp, double hw,
                     long long i, int *col, float *val)
{
    long p, n;
    basis_split(S, i, &p, &n);
    long cnt = 0;
    const uint64_t *bp = &S->sd[0][p * ORW], *bn = &S->sd[1][n * ORW];
    for (long q = p; q < S->nsd[0]; q++) {
        if (S->ncnt[q] == 0) continue;
        uint64_t x[ORW];
        for (int w = 0; w < ORW; w++) x[w] = bp[w] ^ S->sd[0][q * ORW + w];
        int dp = popc_words(x, ORW) / 2;
        if (dp > 2) continue;
        for (long m = S->nbeg[q]; m < S->nbeg[q] + S->ncnt[q]; m++) {
            long long j = S->base[q] + (m - S->nbeg[q]);
            if (j < i) continue;
            for (int w = 0; w < ORW; w++) x[w] = bn[w] ^ S->sd[1][m * ORW + w];
            int dn = popc_words(x, ORW) / 2;
            if (dp + dn > 2) continue;
            if (col) {
                double v;
                if (or_element(S, tbme, esp, hw, i, j, &v) < 0) return -1;
                col[cnt] = (int)j;
                val[cnt] = (float)v;
            }
            cnt++;
        }
    }
    return cnt;
}

/* per-row counts of the half-stored structure (rows i0 .. i1-1) */
int or_count_rows(const or_space *S, long long i0, long long i1, long long *cnt)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (long long i = i0; i < i1; i++) {
        long c = row_walk(S, NULL, NULL, 0.0, i, NULL, NULL);
        if (c < 0) bad = 1;
        cnt[i - i0] = c;
    }
    return bad ? -1 : 0;
}

/* fill rows i0..i1-1 given their local row pointer (rowptr[0] = 0) */
int or_fill_rows(const or_space *S, const float *tbme, const double *esp, double hw,
                 long long i0, long long i1, const long long *rowptr, int *col, float *val)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (long long i = i0; i < i1; i++) {
        long long o = rowptr[i - i0];
        long c = row_walk(S, tbme, esp, hw, i, col + o, val + o);
        if (c != rowptr[i - i0 + 1] - o) bad = 1;
    }
    return bad ? -1 : 0;
}

/* fill an arbitrary list of rows; each row's entries start at off[k] */
int or_fill_row_list(const or_space *S, const float *tbme, const double *esp, double hw,
                     const long long *rows, long nrows, const long long *off, int *col, float *val)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (long k = 0; k < nrows; k++) {
        long c = row_walk(S, tbme, esp, hw, rows[k], col + off[k], val + off[k]);
        if (c != off[k + 1] - off[k]) bad = 1;
    }
    return bad ? -1 : 0;
}

int or_count_row_list(const or_space *S, const long long *rows, long nrows, long long *cnt)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
    for (long k = 0; k < nrows; k++) {
        long c = row_walk(S, NULL, NULL, 0.0, rows[k], NULL, NULL);
        if (c < 0) bad = 1;
        cnt[k] = c;
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* eigensolvers                                                       */
/* ------------------------------------------------------------------ */

/* cyclic Jacobi rotations on a symmetric n x n matrix (row-major, destroyed);
   eigenvalues ascending in w, eigenvectors as columns of V (may be NULL) */
int or_jacobi(int n, double *A, double *w, double *V)
{
    double *Q = V ? V : (double *)malloc(sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; i++) for (int j = 0; j < n; j++) Q[i * n + j] = (i == j);
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; i++) for (int j = 0; j < n; j++) {
            tot += A[i * n + j] * A[i * n + j];
            if (i != j) off += A[i * n + j] * A[i * n + j];
        }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; k++) {          /* A <- A J  (columns p, q) */
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {          /* A <- J^T A (rows p, q) */
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {          /* Q <- Q J */
                    double qkp = Q[k * n + p], qkq = Q[k * n + q];
                    Q[k * n + p] = c * qkp - s * qkq;
                    Q[k * n + q] = s * qkp + c * qkq;
                }
            }
    }
    /* sort ascending */
    int *ord = (int *)malloc(sizeof(int) * n);
    for (int i = 0; i < n; i++) ord[i] = i;
    for (int i = 1; i < n; i++)
        for (int j = i; j > 0 && A[ord[j - 1] * n + ord[j - 1]] > A[ord[j] * n + ord[j]]; j--) {
            int t = ord[j]; ord[j] = ord[j - 1]; ord[j - 1] = t;
        }
    for (int i = 0; i < n; i++) w[i] = A[ord[i] * n + ord[i]];
    if (V) {
        double *tmp = (double *)malloc(sizeof(double) * (size_t)n * n);
        memcpy(tmp, Q, sizeof(double) * (size_t)n * n);
        for (int k = 0; k < n; k++) for (int i = 0; i < n; i++) V[k * n + i] = tmp[k * n + ord[i]];
        free(tmp);
    } else {
        free(Q);
    }
    free(ord);
    return 0;
}

/* y = H x for the half-stored matrix (upper triangle with diagonal) */
static void half_spmv(long long dim, const long long *rowptr, const int *col, const float *val,
                      const double *x, double *y)
{
    memset(y, 0, sizeof(double) * (size_t)dim);
    for (long long i = 0; i < dim; i++)
        for (long long k = rowptr[i]; k < rowptr[i + 1]; k++) {
            long long j = col[k];
            double h = val[k];
            y[i] += h * x[j];
            if (j != i) y[j] += h * x[i];
        }
}

/* number of eigenvalues of the symmetric tridiagonal (alpha, beta) below x:
   the count of negative pivots of the LDL^T factorisation of T - x (Sylvester) */
static int sturm_count(int m, const double *alpha, const double *beta, double x)
{
    int neg = 0;
    double d = 1.0;
    for (int k = 0; k < m; k++) {
        double b2 = k ? beta[k - 1] * beta[k - 1] : 0.0;
        d = alpha[k] - x - (k ? b2 / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) neg++;
    }
    return neg;
}

/* r-th smallest eigenvalue (r = 0, 1, ...) of the tridiagonal by bisection */
static double tridiag_eig(int m, const double *alpha, const double *beta, int r)
{
    double lo = 0.0, hi = 0.0;
    for (int k = 0; k < m; k++) {          /* Gershgorin bounds */
        double rad = (k ? fabs(beta[k - 1]) : 0.0) + (k + 1 < m ? fabs(beta[k]) : 0.0);
        if (k == 0 || alpha[k] - rad < lo) lo = alpha[k] - rad;
        if (k == 0 || alpha[k] + rad > hi) hi = alpha[k] + rad;
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * (fabs(lo) + fabs(hi) + 1e-300); it++) {
        double mid = 0.5 * (lo + hi);
        if (sturm_count(m, alpha, beta, mid) > r) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

/* Lanczos (Sec. 2: repeated matrix-vector products and orthogonalisation)
   with full reorthogonalisation in FP64, started from the given vector.
   Converged when the lowest nev Ritz values move by less than tol (relative)
   in one step.  Writes the lowest nev Ritz values and the lowest Ritz vector
   (the tridiagonal's eigenvector by the Jacobi routine, mapped back). */
int or_lanczos(long long dim, const long long *rowptr, const int *col, const float *val,
               int nev, int max_iter, double tol, const double *v0, double *evals, double *evec0,
               int *iters_out)
{
    int m_max = max_iter < dim ? max_iter : (int)dim;
    if (m_max < 1) return -1;
    double *V = (double *)malloc(sizeof(double) * (size_t)dim * (m_max + 1));
    double *alpha = (double *)calloc(m_max + 1, sizeof(double));
    double *beta = (double *)calloc(m_max + 1, sizeof(double));
    double *w = (double *)malloc(sizeof(double) * (size_t)dim);
    double nrm = 0.0;
    for (long long i = 0; i < dim; i++) nrm += v0[i] * v0[i];
    nrm = sqrt(nrm);
    for (long long i = 0; i < dim; i++) V[i] = v0[i] / nrm;
    double prev[64], cur[64];
    int nprev = 0, m = 0, conv = 0;
    for (int k = 0; k < m_max; k++) {
        half_spmv(dim, rowptr, col, val, &V[(size_t)k * dim], w);
        double a = 0.0;
        for (long long i = 0; i < dim; i++) a += w[i] * V[(size_t)k * dim + i];
        alpha[k] = a;
        for (int pass = 0; pass < 2; pass++)          /* full reorthogonalisation, twice */
            for (int r = 0; r <= k; r++) {
                double h = 0.0;
                for (long long i = 0; i < dim; i++) h += w[i] * V[(size_t)r * dim + i];
                for (long long i = 0; i < dim; i++) w[i] -= h * V[(size_t)r * dim + i];
            }
        double b = 0.0;
        for (long long i = 0; i < dim; i++) b += w[i] * w[i];
        b = sqrt(b);
        beta[k] = b;
        m = k + 1;
        int nv = nev < m ? nev : m;
        if (nv > 64) nv = 64;
        for (int r = 0; r < nv; r++) cur[r] = tridiag_eig(m, alpha, beta, r);
        if (m >= nev && nprev == nv) {
            double d = 0.0;
            for (int r = 0; r < nv; r++) {
                double e = fabs(cur[r] - prev[r]) / (fabs(cur[r]) > 1.0 ? fabs(cur[r]) : 1.0);
                if (e > d) d = e;
            }
            if (d < tol) conv = 1;
        }
        for (int r = 0; r < nv; r++) prev[r] = cur[r];
        nprev = nv;
        if (b < 1e-12 * (fabs(a) + 1.0)) conv = 1;      /* invariant subspace: exact */
        if (conv || m == m_max) break;
        for (long long i = 0; i < dim; i++) V[(size_t)(k + 1) * dim + i] = w[i] / b;
    }
    int nv = nev < m ? nev : m;
    for (int r = 0; r < nv; r++) evals[r] = prev[r];
    for (int r = nv; r < nev; r++) evals[r] = NAN;
    if (evec0) {
        double *T = (double *)calloc((size_t)m * m, sizeof(double));
        double *ev = (double *)malloc(sizeof(double) * m);
        double *Y = (double *)malloc(sizeof(double) * (size_t)m * m);
        for (int r = 0; r < m; r++) {
            T[r * m + r] = alpha[r];
            if (r + 1 < m) { T[r * m + r + 1] = beta[r]; T[(r + 1) * m + r] = beta[r]; }
        }
        or_jacobi(m, T, ev, Y);
        for (long long i = 0; i < dim; i++) {
            double s = 0.0;
            for (int r = 0; r < m; r++) s += V[(size_t)r * dim + i] * Y[r * m + 0];
            evec0[i] = s;
        }
        free(T); free(ev); free(Y);
    }
    if (iters_out) *iters_out = m;
    free(V); free(alpha); free(beta); free(w);
    return conv ? 0 : 1;
}

/* dense H (row-major) by or_element over every (i, j): tiny bases only */
int or_dense_sc(const or_space *S, const float *tbme, const double *esp, double hw, double *H)
{
    long long D = S->dim;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : bad)
    for (long long i = 0; i < D; i++)
        for (long long j = 0; j < D; j++) {
            double v;
            if (or_element(S, tbme, esp, hw, i, j, &v) < 0) bad = 1;
            H[i * D + j] = v;
        }
    return bad ? -1 : 0;
}

/* tridiagonal eigenvalue by bisection, exposed for its own pin */
/* y = H x for a half-stored matrix (the product Lanczos applies, Sec. 2) */
int or_half_spmv(long long dim, const long long *rowptr, const int *col, const float *val, const double *x,
                 double *y)
{
    if (dim < 0 || (dim > 0 && (!rowptr || !x || !y))) return -1;
    half_spmv(dim, rowptr, col, val, x, y);
    return 0;
}

double or_tridiag_eig(int m, const double *alpha, const double *beta, int r)
{
    return tridiag_eig(m, alpha, beta, r);
}

/* ------------------------------------------------------------------ */
/* gradient of the lowest eigenvalue                                   */
/* ------------------------------------------------------------------ */

/* Hellmann-Feynman: dE0/dt = <psi| dH/dt |psi>.  Over the half-stored
   structure: every stored (i,j) whose value uses parameter t with sign s adds
   w * s * psi_i * psi_j, w = 2 off the diagonal (the mirrored element) and 1 on
   it.  The terms are found with the same Slater-Condon cases as or_element. */
int or_grad_elementwise(const or_space *S, const long long *rowptr, const int *col,
                        const double *psi, double *grad)
{
    memset(grad, 0, sizeof(double) * (size_t)S->tbme_len);
    uint64_t oi[ORCW], oj[ORCW], x[ORCW];
    for (long long i = 0; i < S->dim; i++) {
        state_occ(S, i, oi);
        for (long long k = rowptr[i]; k < rowptr[i + 1]; k++) {
            long long j = col[k];
            state_occ(S, j, oj);
            double f = (j == i ? 1.0 : 2.0) * psi[i] * psi[j];
            int nd = 0;
            for (int w = 0; w < ORCW; w++) { x[w] = oi[w] ^ oj[w]; nd += __builtin_popcountll(x[w]); }
            nd /= 2;
            int sg;
            long long idx;
            if (nd == 0) {
                for (int a = 0; a < S->ntot; a++) {
                    if (!occ_bit(oj, a)) continue;
                    for (int b = a + 1; b < S->ntot; b++) {
                        if (!occ_bit(oj, b)) continue;
                        idx = or_tbme_index(S, a, b, a, b, &sg);
                        if (idx < 0) return -1;
                        grad[idx] += sg * f;
                    }
                }
                continue;
            }
            int in_i[2] = {0, 0}, in_j[2] = {0, 0}, ni = 0, nj = 0;
            for (int q = 0; q < S->ntot; q++) {
                if (occ_bit(x, q) && occ_bit(oi, q)) in_i[ni++] = q;
                if (occ_bit(x, q) && occ_bit(oj, q)) in_j[nj++] = q;
            }
            uint64_t t[ORCW];
            memcpy(t, oj, sizeof(t));
            if (nd == 1) {
                int a = in_i[0], c = in_j[0];
                int s = annihilate(t, c);
                s *= create(t, a);
                for (int q = 0; q < S->ntot; q++) {
                    if (!occ_bit(oj, q) || q == c) continue;
                    idx = or_tbme_index(S, a, q, c, q, &sg);
                    if (idx < 0) return -1;
                    grad[idx] += s * sg * f;
                }
            } else {
                int a = in_i[0], b = in_i[1], c = in_j[0], d = in_j[1];
                int s = annihilate(t, c);
                s *= annihilate(t, d);
                s *= create(t, b);
                s *= create(t, a);
                idx = or_tbme_index(S, a, b, c, d, &sg);
                if (idx < 0) return -1;
                grad[idx] += s * sg * f;
            }
        }
    }
    return 0;
}

// Internal data layout of libcih (host and device).  Not part of the ABI.
#pragma once

#include <cstdint>
#include <string>
#include <exception>
#include <functional>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "cih.h"

namespace cih {

constexpr int kMaxWords = 4;              // <= 256 orbitals per species
constexpr int kSortTile = 4096;           // longest neighbour list the sort handles

// ---------------------------------------------------------------- device view

// One species' sub-determinant tables and neighbour lists.
struct DevSpecies {
    const uint64_t *bits;      // n_sd x W words (W = basis word count)
    const int8_t *N;           // oscillator quanta of each sub-det
    const int32_t *cls_end;    // per sub-det: one past the end of its (2M, parity) class
    const int64_t *fw_off;     // n_sd + 1: forward same-class neighbours (1 or 2 moves)
    const int32_t *fw;         //   sorted ascending, all > x
    const int64_t *n1_off;     // n_sd + 1: every one-move neighbour
    const int32_t *n1;         //   sorted ascending
    const int64_t *n1_later;   // per sub-det: first one-move entry beyond its own class
    int32_t n_sd;
    int32_t n_orb;
    int32_t orb_base;          // combined index of this species' orbital 0
};

// Everything the Hamiltonian kernels read.
struct DevBasis {
    DevSpecies sp[2];          // 0 = protons, 1 = neutrons
    const int32_t *nb;         // per proton sub-det: first neutron partner
    const int32_t *nc;         //   number of partners
    const int64_t *rowbase;    // n_p + 1: first row of each proton sub-det
    const int8_t *orbN;        // combined orbital -> N
    const int32_t *pid;        // ntot x ntot pair id (see pair_code), -1 = none
    const int32_t *gsize;      // per global group: pairs in the group
    const int64_t *goff;       // per global group: table offset of its triangle
    int32_t ngroups;           // global groups of the table layout
    int32_t n_p;
    int32_t ntot;
    int64_t dim;
    int64_t tbme_len;
    // fast paths
    const int32_t *fw_tb[2];   // per forward entry: two-move table index << 1 | sign, or -1
    const uint32_t *n1_info;   // per neutron one-move entry: packed move (see neighbours.cu)
    const int16_t *pn_S;       // n_orb_p x pn_G
    const int32_t *pn_gsize;   // pn_G
    const int32_t *pn_goff;    // pn_G
    const int8_t *m2p;         // proton orbital 2m
    const int8_t *Np;          // proton orbital N
    int32_t pn_G;
    int32_t pn_m2span;
    int32_t max_cand;          // largest candidate list of a proton sub-det
    int *queue;                // work counter (unused by the row kernels)
    // candidate table: for proton sub-det p, records cand_off[p] .. cand_off[p+1]
    // (later same-class sub-dets with one or two protons moved, then later-class
    // sub-dets with one proton moved, ascending), one int4 each:
    //   x  column base rowbase[q] - nbeg[q]
    //   y  directory indices of q's neutron range: start | end << 16
    //   z  one-move: S row bases A_u | A_v << 16; two-move: table index << 1 | sign
    //   w  bits 0..7 K_a, 8 N_a & 1, 9 sign, 16..23 a, 24..31 c (one-move only)
    const int64_t *cand_off;
    const int4 *cand;
    const uint8_t *cand_self;      // per record: 0 if n can never lie in q's range,
                                   // else 1 + the largest N of a partner; bit 7 = two-move
    const int32_t *row_p;          // row -> proton sub-det
    int32_t A;                     // particles
    int32_t nZ[2];                 // particles per species
    // neutron one-move lists packed (neighbour, move info), and their bucket
    // directory: for neutron n, dir[n * dir_len + 1 + rc * NL + L] = number of
    // entries of n's one-move list in buckets <= (relative class rc, level L);
    // dir[n * dir_len] = 0.  rc = ((2M_y - 2M_n + DM) / 2) * 2 + (N_y & 1).
    const int2 *n1p;
    const int16_t *dir;
    int32_t dir_len, NL, DM;
    // count lists: per proton sub-det p, the directory positions its one-move
    // candidates' segments start and end at, with multiplicities (position,
    // coefficient), and the number of candidates whose range holds n itself
    // per N_n
    const int64_t *clist_off;  // n_p + 1, or null when the count walks the candidates
    const int2 *clist;
    const uint16_t *cself_sfx; // n_p x NL
    const int16_t *self_rel;       // per neutron n: entries of its one-move list below n
    const uint8_t *occ[2];         // per sub-det: its occupied orbitals, ascending (Z_s each)
    // one-body table layout (see OneBodyLayout)
    const int16_t *ob_grp, *ob_loc;
    const int32_t *ob_gsize, *ob_goff;
};

// pid entry: bits 0..15 local pair index u, bits 16..27 global group id,
// bit 30 set when the orbitals are given in descending order (sign -1).
__host__ __device__ inline int32_t pair_code(int group, int u, bool swapped)
{
    return (group << 16) | u | (swapped ? (1 << 30) : 0);
}

// device tables of one species used while building the neighbour lists
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
    const int32_t *hash;        // open-addressing table of sub-det indices, -1 = empty
    uint32_t hash_mask;         // capacity - 1 (power of two)
    const uint64_t *bitsT;      // W x n_sd: the bit strings word-major (coalesced scans)
    const int32_t *orb_upto;    // [N]: orbitals with shell <= N (orbitals are ordered by shell)
    int32_t maxN;               // highest orbital shell
};

// ---------------------------------------------------------------- host side

struct Species {
    int Z = 0;
    int n_orb = 0;
    int N0 = 0, NF = -1;
    int Nsub_max = 0;
    std::vector<int> oN, ol, oj2, om2;       // orbital quantum numbers
    int64_t n_sd = 0;
    std::vector<uint64_t> bits;               // n_sd x kMaxWords
    std::vector<int> N, M2;                   // per sub-det
    std::vector<int> cls;                     // class id per sub-det
    std::vector<int> cls_M2, cls_par, cls_begin, cls_end;
};

struct Layout {
    // per channel (pp, nn, pn): pairs grouped, group metadata
    int64_t chan_len[3] = {0, 0, 0};
    int64_t total = 0;
    std::vector<int32_t> gsize;               // global group id -> size
    std::vector<int64_t> goff;                // global group id -> table offset
    std::vector<int32_t> pid;                 // ntot x ntot
};

// One-body table layout: per species, groups of orbitals with equal (2m, N
// parity) in the order (species, 2m, parity), members ascending; each group
// stores its packed upper triangle (a <= c).
struct OneBodyLayout {
    int64_t total = 0;
    std::vector<int16_t> grp, loc;            // per combined orbital: group, place in it
    std::vector<int32_t> gsize, goff;         // per group
};

// pn pair index split u(a, b) = S[a][kappa] + r(b): kappa = dense group key
// ((2m_a + 2m_b + m2span) / 2) * 2 + ((N_a + N_b) & 1), r(b) = number of lower
// neutron orbitals with the same 2m and N parity as b.  Groups absent from the
// table have size 0.
struct PnSplit {
    int G = 0;                                // dense group keys
    int m2span = 0;                           // largest |2m_a + 2m_b|
    std::vector<int16_t> S;                   // n_orb_p x G
    std::vector<int32_t> gsize, goff;         // per dense key
    std::vector<int32_t> rn;                  // per neutron orbital
};

struct DevBuffers {
    std::vector<void *> owned;                // every cudaMalloc made for the handle
};

}  // namespace cih

struct cih_basis {
    cih_space_t space{};
    int W = 1;                                // words per bit string (1, 2 or 4)
    int N0tot = 0, Nlim = 0;
    cih::Species s[2];
    int64_t dim = 0;
    std::vector<int32_t> nb, nc;
    std::vector<int64_t> rowbase;
    cih::Layout layout;
    cih::OneBodyLayout onebody;
    cih::PnSplit pn;
    cih::SpeciesBuild sbuild[2]{};
    cih::DevBasis dev{};
    cih::DevBuffers buffers;
    int64_t *scan_scratch = nullptr;          // block sums of the row-pointer scan
    int64_t scan_scratch_len = 0;
    int *dev_status = nullptr;                // kernel error word
    int device = 0;
    cudaMemPool_t pool = nullptr;             // library pool the handle's buffers come from
    cudaStream_t stream = nullptr;            // stream of the build
    int launch_warps = 16;                    // row kernels: warps per CTA (8 or 16)
    int launch_ctas = 0;                      // row kernels: CTAs per SM (0 = as many as fit)
    int count_walk = 0;                       // count pass: 1 = walk the candidates even with count lists
};

namespace cih {

// f0() here and f1() on a second thread; an exception of either is rethrown
template <class F0, class F1>
inline void side_by_side(F0 &&f0, F1 &&f1)
{
    std::exception_ptr e1;
    std::thread th([&]() {
        try {
            f1();
        } catch (...) {
            e1 = std::current_exception();
        }
    });
    try {
        f0();
    } catch (...) {
        th.join();
        throw;
    }
    th.join();
    if (e1) std::rethrow_exception(e1);
}

// every kernel launch site adds the launches it makes (capi.cpp)
void count_launches(int64_t n);

// the library's device memory pool of a device (keeps freed memory for reuse)
int device_pool(int device, cudaMemPool_t *pool);

// phase timer printed to stderr when the environment sets CIH_TIMING
struct Timer {
    const char *what;
    double t0;
    explicit Timer(const char *w);
    ~Timer();
    void mark(const char *phase);
    void mark_sync(const char *phase, cudaStream_t st);   // synchronises st only when timing is on
};

// error reporting (capi.cpp)
int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// host basis construction (basis.cpp)
int build_host_basis(const cih_space_t &sp, cih_basis &b);
// the same in two parts: orbitals, sub-determinants and classes; then partner
// ranges, table layout and pn split (which the first device passes do not need)
int build_host_species(const cih_space_t &sp, cih_basis &b);
int build_host_rest(cih_basis &b);

// device set-up (neighbours.cu)
// device set-up after build_host_species; host_rest() (build_host_rest) runs
// while the first device passes are in flight
int upload_and_build_neighbours(cih_basis &b, cudaStream_t st, const std::function<int()> &host_rest);

// kernels (ham.cu)
int launch_count(const cih_basis &b, int64_t *rowptr, cudaStream_t st);
int launch_scan(const cih_basis &b, int64_t *rowptr, cudaStream_t st);
// interleaved: tables element-major (len x K); em: values element-major (nnz x K)
// sharded: col / val hold only rows r0 .. r1 - 1 (positions relative to rowptr[r0]);
// t1: a one-body table (OneBodyLayout) in place of the orbital energies, or null
int launch_fill(const cih_basis &b, const int64_t *rowptr, int K, double hw, const float *tbme, bool interleaved, bool em,
                const double *esp, int32_t *col, float *val, cudaStream_t st, int64_t r0 = 0, int64_t r1 = -1,
                bool sharded = false, const double *t1 = nullptr);
int launch_interleave(int K, int64_t len, const float *in, float *out, cudaStream_t st);
// one-time set-up of the row kernels a call with K sets would launch (shared-
// memory limits), so that launches made during a stream capture only launch
int prepare_rows(const cih_basis &b, int K);
int launch_grad(const cih_basis &b, const int64_t *rowptr, int K, const double *psi,
                unsigned long long *acc, cudaStream_t st);
int launch_grad_finish(int64_t n, const unsigned long long *acc, double *grad, cudaStream_t st);

// generic device scans (scan.cu)
int exclusive_scan_i64(int64_t *data, int64_t n, int64_t *block_sums, int64_t block_sums_len,
                       cudaStream_t st);
int64_t scan_scratch_needed(int64_t n);

// symmetric tridiagonal eigenproblem, ascending, Z row-major n x n (tridiag.cpp)
void tridiag_qr(int n, std::vector<double> &d, std::vector<double> e, std::vector<double> &Z);
// the same eigenvalues with only the last component of each eigenvector
void tridiag_qr_last(int n, std::vector<double> &d, std::vector<double> e, std::vector<double> &zlast);
// normalised eigenvector for an eigenvalue by inverse iteration
void tridiag_eigenvector(int n, const double *d, const double *e, double theta, double *z);

// Lanczos (lanczos.cu)
// A row shard's part of a Lanczos run over several processes: its rows, the
// whole matrix's squared strictly-upper Frobenius norm (summed over the
// shards), and two caller buffers (dim x K, zero on entry) that `combine`
// sums over the shards in place after each product.
struct ShardRun {
    int64_t r0 = 0, r1 = 0;
    double f2 = 0.0;
    unsigned long long *acc = nullptr;
    double *yx = nullptr;
    int (*combine)(void *ctx) = nullptr;
    void *ctx = nullptr;
};
int lanczos(const cih_basis &b, const int64_t *rowptr, const int32_t *col, const float *val,
            int K, int nev, int max_iter, double tol, double *evals, double *evec0, cudaStream_t st,
            bool values_em = false, const ShardRun *sh = nullptr);
// the sum of squares of the strictly-upper values of rows [r0, r1) (all K
// sets), the arrays starting at rowptr[r0]: one shard's part of the bound
int upper_sumsq(const cih_basis &b, const int64_t *rowptr, int64_t r0, int64_t r1, const float *val, int K,
                bool values_em, double *f2, cudaStream_t st);
// device bytes lanczos() allocates for a call
int64_t lanczos_bytes(int64_t dim, int64_t nnz, int K, int max_iter);
// y = H x for K sets from the stored upper half (x, y element-major: x[i * K + s])
int ham_spmv(const cih_basis &b, const int64_t *rowptr, const int32_t *col, const float *val, int K, bool values_em,
             const double *x, double *y, cudaStream_t st);

// tables from host memory, matrix to host memory, copies overlapped (host_io.cpp)
int build_host(cih_basis &b, int K, double hw, const float *tbme_h, const double *esp_h, int64_t *rowptr_h,
               int32_t *col_h, float *val_h, int64_t capacity, int64_t *nnz_out, cudaStream_t st);

// count, admission, build, Lanczos and adjoint of a batch (batch.cpp)
int batch_solve(cih_instance_t *inst, int n, double hw, int nev, int max_iter, double tol, int64_t budget,
                cudaStream_t st);

}  // namespace cih

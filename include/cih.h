/*
 * cih.h -- C ABI of libcih: GB300 (sm_103a) construction of the half-stored
 * M-scheme configuration-interaction Hamiltonian.
 *
 * The method is that of arXiv 1412.5989 ("Accelerating Ab Initio Nuclear
 * Physics Calculations with GPUs"): the nuclear many-body Schroedinger
 * equation becomes a large sparse symmetric matrix eigenproblem over a basis
 * of Slater determinants (Sec. 1); its nonzeros are located, computed and
 * stored, only half of the symmetric matrix being generated (Sec. 2); the
 * nonzeros are counted in one pass so the arrays can be allocated and then
 * computed in a second pass (Sec. 4.1), stored in compressed-row form
 * (Sec. 4.1); and the lowest eigenpairs follow by Lanczos (Sec. 2).
 *
 * Conventions (the paper states them in prose only; these are the readings
 * this library implements, identical to the CPU oracle's):
 *   - orbitals of a species with Z > 0 particles: harmonic-oscillator states
 *     (N, l, 2j, 2m) with N <= N_F + Nmax, N_F the highest shell filled by the
 *     lowest configuration, ordered (N, l, 2j, 2m) ascending; a species with
 *     no particles has no orbitals.  Combined index: protons 0..n_orb_p-1,
 *     then neutrons n_orb_p..n_orb_p+n_orb_n-1.
 *   - sub-determinants of a species: its particle subsets that occur in at
 *     least one basis state, ordered by (2M, N mod 2, N, bit string read as
 *     an unsigned multiword integer) ascending.
 *   - basis: pairs (proton sub-det p, neutron sub-det n) with 2M_p + 2M_n =
 *     2M, N_p + N_n <= N0 + Nmax and N_p + N_n = N0 + Nmax (mod 2), in
 *     lexicographic (p, n) order.  Each p's partners form one contiguous range.
 *   - |Phi> = a+_{i1} ... a+_{iA} |0>, i1 < ... < iA (combined index).
 *   - H = sum_a e_a a+_a a_a + sum_{a<b, c<d} V_{ab,cd} a+_a a+_b a_d a_c,
 *     e_a = hbar_omega (N_a + 3/2) unless a per-orbital table is given.
 *   - stored: the upper triangle j >= i of every (i, j) whose determinants
 *     differ by at most two particles, whatever the value (so K tables share
 *     one structure); rows in basis order, columns ascending.
 *   - two-body table (input format), one set = tbme_len floats: channels pp,
 *     nn, pn concatenated; a pair (a<b) is in its channel when N_a + N_b <=
 *     N0 + Nmax - N0(other A-2 particles); pairs grouped by (2M_pair, parity)
 *     ascending, lexicographic (a, b) inside a group; each group stores its
 *     packed row-major upper triangle (bra pair index u <= ket pair index v at
 *     group_offset + u*n - u(u-1)/2 + (v-u)).  One entry stands for V_{ab,cd}
 *     and V_{cd,ab}; a swapped pair flips the sign.
 *
 * Ownership: the caller owns every device array passed in (allocate it with
 * any allocator, e.g. torch).  The library owns the basis handle and the
 * device memory behind it (sub-determinant tables, neighbour lists, table
 * layout, scan scratch).  Every call is ordered on the given CUDA stream
 * (a cudaStream_t passed as void*; NULL = the legacy default stream).  Calls
 * that return a host value (nnz_out, evals_host) synchronise that stream.
 * A handle must not be used by two host threads at once.  The library keeps
 * per-device state for the life of the process (its memory pool, the device
 * address of cih_rowptr_scan_static's array); resetting a device after the
 * library has used it is not supported.
 *
 * Errors: every call returns 0 or a negative CIH_ERR_* code; no C++ exception
 * crosses the ABI.  cih_strerror() names a code; cih_last_error_detail()
 * returns the last failure's message for the calling thread.
 */
#ifndef CIH_H
#define CIH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CIH_OK              0
#define CIH_ERR_ARG        -1   /* invalid argument or NULL pointer          */
#define CIH_ERR_NOMEM      -2   /* a library-owned allocation failed         */
#define CIH_ERR_CAPACITY   -3   /* the result does not fit (e.g. nnz budget) */
#define CIH_ERR_TIMEOUT    -4   /* a bounded device wait gave up             */
#define CIH_ERR_UNSUPPORTED -5  /* a size outside what the kernels handle    */
#define CIH_ERR_CUDA       -6   /* a CUDA runtime call failed                */
#define CIH_ERR_DEVICE     -7   /* a kernel's own bounds check tripped        */

typedef struct {
    int32_t Z;      /* protons                                 */
    int32_t N;      /* neutrons                                */
    int32_t Nmax;   /* oscillator quanta above the lowest configuration */
    int32_t twoM;   /* twice the total angular-momentum projection      */
} cih_space_t;

typedef struct cih_basis *cih_basis_h;

/* Build the many-body basis for *space on the current CUDA device (Sec. 2:
 * the index tables that define the basis come before the matrix): orbitals,
 * sub-determinants of both species, partner ranges, row offsets, the
 * two-body table layout, and the neighbour lists the kernels walk.  Work is
 * ordered after `stream`'s earlier work; the neutron half of the list passes
 * runs on a second, library-created stream that joins `stream` before the
 * call returns, and the call returns after both have finished.
 * *out receives a new handle (release with cih_basis_destroy).
 * Errors: CIH_ERR_ARG (NULL, Z or N < 0, Nmax < 0), CIH_ERR_UNSUPPORTED
 * (more than 256 orbitals per species, a dimension above 2^31-1, a
 * neighbour list longer than the sort tile), CIH_ERR_NOMEM, CIH_ERR_CUDA. */
int cih_basis_enumerate(const cih_space_t *space, cih_basis_h *out, void *stream);

/* Sizes of a basis.  Any output pointer may be NULL.
 * dim: basis dimension (rows); n_orb_p / n_orb_n: orbitals per species;
 * tbme_len[3]: entries of the pp, nn and pn channels (one set's table is
 * their sum); n_sd[2]: sub-determinants per species. */
int cih_basis_info(cih_basis_h h, int64_t *dim, int32_t *n_orb_p, int32_t *n_orb_n,
                   int64_t tbme_len[3], int64_t n_sd[2]);

/* Copy host-side basis tables out (for inspection and tests).  Any pointer
 * may be NULL.  orbitals: (n_orb_p + n_orb_n) x 4 int32 (N, l, 2j, 2m);
 * subdet_bits_p / _n: n_sd x 4 uint64 words (bit k = species orbital k);
 * nbeg / ncnt: per proton sub-det neutron partner range; rowbase: n_sd_p + 1
 * first-row offsets. */
int cih_basis_tables(cih_basis_h h, int32_t *orbitals, uint64_t *subdet_bits_p,
                     uint64_t *subdet_bits_n, int32_t *nbeg, int32_t *ncnt, int64_t *rowbase);

int cih_basis_destroy(cih_basis_h h);

/* Host tables only, no device work: the same basis and table layout as
 * cih_basis_enumerate, for inspection and for checking the host logic on a
 * machine without a GPU.  Only cih_basis_info, cih_basis_tables,
 * cih_tbme_index and cih_basis_destroy accept such a handle; the device
 * calls return CIH_ERR_ARG.  Errors as cih_basis_enumerate. */
int cih_basis_host_only(const cih_space_t *space, cih_basis_h *out);

/* Table index of V_{ab,cd} for combined orbitals a, b, c, d in any order
 * (the layout above): *index = -1 and *sign = 0 when the pairs are not one
 * table entry, else *sign = +-1 from the pair orders.  Host-side lookup. */
int cih_tbme_index(cih_basis_h h, int32_t a, int32_t b, int32_t c, int32_t d,
                   int64_t *index, int32_t *sign);

/* Count pass + scan (Sec. 4.1: a first pass over the nonzeros only counts
 * them, so that the output arrays can be sized).  Writes the exclusive prefix sum
 * of the per-row counts of the half-stored structure into rowptr_dev
 * (device, dim + 1 int64, caller-owned): rowptr[0] = 0, rowptr[dim] = nnz.
 * If nnz_out != NULL the stream is synchronised and *nnz_out = nnz.
 * Errors: CIH_ERR_ARG, CIH_ERR_CUDA. */
int cih_ham_count(cih_basis_h h, int64_t *rowptr_dev, int64_t *nnz_out, void *stream);

/* Fill pass (Sec. 2 and 4.1: the second pass finds each nonzero again,
 * computes it and stores it): with rowptr_dev from cih_ham_count, write for every stored
 * nonzero its column (col_dev: nnz int32) and, for each of the K two-body
 * sets, its value (val_dev: K x nnz float, set-major).
 *   tbme_dev: K x tbme_len float (device), set-major, layout above;
 *   e_sp_dev: NULL for e_a = hbar_omega (N_a + 3/2), else (n_orb_p +
 *             n_orb_n) double one-body energies (device, combined index).
 * Values: single-term elements (two-particle moves) are the table entry
 * times +-1, exactly.  Multi-term elements (the diagonal, one-particle moves)
 * are sums of FP32 terms (one-body energies, table entries) carried as
 * double-float pairs (hi + lo, about 48 significant bits), rounded once to
 * FP32.  For the few dozen terms of one element this is the exact sum in all
 * but pathological cancellations, so the stored value agrees with the FP64
 * sum rounded to FP32 within 1e-5 (|value| + 1) (in practice bit for bit).
 * Errors: CIH_ERR_ARG (K < 1, NULL arrays), CIH_ERR_CUDA. */
int cih_ham_fill(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, double hbar_omega,
                 const float *tbme_dev, const double *e_sp_dev,
                 int32_t *col_dev, float *val_dev, void *stream);

/* One-body table (Sec. 2: MFDn reads its one-body operator, the kinetic
 * energy, from file): with it, H = sum_{a,c} t_ac a+_a a_c + the two-body
 * part, in place of the orbital energies e_a.  t is symmetric and has entries
 * only for orbitals a, c of one species with equal 2m and equal N parity
 * (Delta N = 2 couplings included).  Layout: per species (protons first),
 * groups of such orbitals ordered by (2m, parity) ascending, members in
 * ascending orbital order; a group stores its packed row-major upper triangle
 * (u <= v at group_offset + u*n - u(u-1)/2 + (v-u)), one double each.
 * cih_onebody_info: *len = entries of the table.
 * cih_onebody_index: *index of t_ac for combined orbitals a, c in either
 * order, -1 if a and c are not one group.  Host-side; any handle.
 * Errors: CIH_ERR_ARG (NULL). */
int cih_onebody_info(cih_basis_h h, int64_t *len);
int cih_onebody_index(cih_basis_h h, int32_t a, int32_t c, int64_t *index);

/* As cih_ham_fill with a one-body table (layout above; onebody_dev: len
 * double, device, shared by the K sets) in place of the orbital energies:
 * the diagonal holds sum over occupied a of t_aa plus the two-body pairs, and
 * a one-particle move a <- c holds its sign times (t_ac + the spectator sum).
 * Values and their summation as cih_ham_fill.  Errors as cih_ham_fill. */
int cih_ham_fill_onebody(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, const float *tbme_dev,
                         const double *onebody_dev, int32_t *col_dev, float *val_dev, void *stream);

/* Row-sharded fill (Sec. 2 and 4.1: the matrix is split into row chunks of
 * about equal nonzero counts, one per process): the fill of rows r0 .. r1 - 1
 * only, written to arrays that hold just those rows.  With nnz_s =
 * rowptr[r1] - rowptr[r0], stored nonzero e of those rows goes to
 * col_dev[e - rowptr[r0]] (nnz_s int32) and its value for set k to
 * val_dev[k * nnz_s + e - rowptr[r0]] (K x nnz_s float).  rowptr_dev is the
 * whole row-pointer array from cih_ham_count (device, dim + 1 int64); the
 * other arguments as cih_ham_fill.  The shards of any partition of 0 .. dim
 * concatenate to cih_ham_fill's arrays bit for bit.  0 <= r0 <= r1 <= dim;
 * r0 == r1 does nothing.  Errors: CIH_ERR_ARG, CIH_ERR_CUDA. */
int cih_ham_fill_rows(cih_basis_h h, const int64_t *rowptr_dev, int64_t r0, int64_t r1, int32_t K,
                      double hbar_omega, const float *tbme_dev, const double *e_sp_dev, int32_t *col_dev,
                      float *val_dev, void *stream);

/* Row boundaries of nshards shards of about equal stored nonzeros (Sec. 4.1's
 * balancing of chunks by nonzero count), from a host copy of the row pointers
 * (rowptr_host: dim + 1 int64): bounds_host[0] = 0 <= bounds_host[1] <= ... <=
 * bounds_host[nshards] = dim (nshards + 1 int64, host); shard k is rows
 * bounds[k] .. bounds[k + 1] - 1, starting at the first row whose elements
 * begin at or after k/nshards of the nonzeros.  Host only.
 * Errors: CIH_ERR_ARG. */
int cih_shard_rows(const int64_t *rowptr_host, int64_t dim, int32_t nshards, int64_t *bounds_host);

/* As cih_ham_fill, with the K tables interleaved element-major
 * (tbme_il_dev[t * K + k] = entry t of set k; see cih_tbme_interleave), so that
 * the K values of one nonzero come from one contiguous read.  Output layout as
 * cih_ham_fill (values set-major).  Errors as cih_ham_fill. */
int cih_ham_fill_interleaved(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, double hbar_omega,
                             const float *tbme_il_dev, const double *e_sp_dev,
                             int32_t *col_dev, float *val_dev, void *stream);

/* The batched fill: K interleaved tables in (tbme_il_dev[t * K + k], as from
 * cih_tbme_interleave) and the values out element-major: val_em_dev[e * K +
 * k] is the value of stored nonzero e in set k (nnz x K float, device,
 * caller-owned), so each nonzero's K values are one contiguous write.  This
 * is the layout cih_lanczos_lowest_em reads.  Columns as cih_ham_fill.
 * Multi-term values (diagonal, one-particle moves) are summed per set in term
 * order, so they can differ from the K = 1 fill in the last bit; single-term
 * values are identical.  Errors as cih_ham_fill. */
int cih_ham_fill_batched(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, double hbar_omega,
                         const float *tbme_il_dev, const double *e_sp_dev, int32_t *col_dev, float *val_em_dev,
                         void *stream);

/* End to end with host memory (Sec. 2 and 4.1 as cih_ham_count + cih_ham_fill,
 * with the host copies inside the call): the K two-body tables are copied
 * host -> device, the count pass and scan run, the row pointers come back
 * (one synchronisation, which gives nnz), then the fill runs in 8 row chunks
 * of about equal nonzero counts while a second stream copies each finished
 * chunk's columns and values device -> host.
 *   tbme_host: K x tbme_len float (set-major); e_sp_host: NULL or
 *   n_orb_p + n_orb_n double; rowptr_host: dim + 1 int64; col_host:
 *   capacity int32; val_host: K x capacity float, the values of set k at
 *   val_host[k * capacity + e]; *nnz_out (may be NULL): stored nonzeros.
 * Host arrays should be page-locked (cudaHostAlloc, cudaHostRegister, a
 * pinned torch tensor): then the copies run at link speed and overlap the
 * fill; pageable memory works, but each copy then waits for its data.
 * Device scratch (tables, row pointers, columns, K x values) is
 * library-allocated for the call.  Synchronises `stream`.
 * Errors: CIH_ERR_ARG; CIH_ERR_CAPACITY when nnz > capacity (rowptr_host and
 * *nnz_out are written, nothing else); CIH_ERR_NOMEM; CIH_ERR_CUDA. */
int cih_ham_build_host(cih_basis_h h, int32_t K, double hbar_omega, const float *tbme_host, const double *e_sp_host,
                       int64_t *rowptr_host, int32_t *col_host, float *val_host, int64_t capacity, int64_t *nnz_out,
                       void *stream);

/* tbme_il_dev[t * K + k] = tbme_dev[k * tbme_len + t] (device arrays, caller-
 * owned, stream-ordered).  Errors: CIH_ERR_ARG, CIH_ERR_CUDA. */
int cih_tbme_interleave(int32_t K, int64_t tbme_len, const float *tbme_dev, float *tbme_il_dev, void *stream);

/* Launch shape of the row kernels (count, fill, adjoint) of this handle:
 * warps_per_cta 8 or 16, ctas_per_sm 0 (as many as fit) or a cap.
 * Errors: CIH_ERR_ARG. */
int cih_set_launch(cih_basis_h h, int32_t warps_per_cta, int32_t ctas_per_sm);

/* Which form of the count pass (Sec. 4.1's first pass) cih_ham_count runs for
 * this handle: walk = 0 (default) sums each row's segment lengths from the
 * per-proton count lists where the basis has them (bucket directories of at
 * most 4096 entries and at most 63 oscillator levels) and walks the
 * candidates otherwise; walk = 1 always walks the candidates, the same walk
 * the fill makes.  Both give the same row pointers.  Errors: CIH_ERR_ARG. */
int cih_set_count_mode(cih_basis_h h, int32_t walk);

/* Autotuner: times the fill (cih_ham_fill; cih_ham_fill_interleaved when
 * interleaved == 1; cih_ham_fill_batched when interleaved == 2; same
 * arguments) for every launch shape -- warps per CTA in
 * {16, 8} x CTAs per SM in {as many as fit, 1, 2, 3} -- with CUDA events
 * (best of two after one warm-up), keeps the fastest on the handle and reports
 * it.  The outputs col_dev / val_dev are written (with the final, correct
 * values).  Synchronises `stream`.  Errors as cih_ham_fill. */
int cih_autotune_fill(cih_basis_h h, const int64_t *rowptr_dev, int32_t K, double hbar_omega,
                      const float *tbme_dev, int32_t interleaved, const double *e_sp_dev,
                      int32_t *col_dev, float *val_dev, void *stream,
                      int32_t *best_warps, int32_t *best_ctas, float *best_ms);

/* Lowest eigenpairs by Lanczos (Sec. 2) for each of K matrices sharing one
 * structure (the output of one cih_ham_fill call): FP32 half-stored values,
 * FP64 vectors and matrix-vector accumulation, FP64 full reorthogonalisation
 * (classical Gram-Schmidt twice per step), FP64 tridiagonal eigenvalues by
 * implicit QR on the host.  All K Krylov sequences advance together; a set whose
 * nev residual bounds beta_m |z_m| meet tol * max(1, |theta|) stops there.
 *   val_dev: K x nnz float (set-major); 1 <= K <= 256; nev <= 64: eigenvalues
 *   wanted; max_iter <= 2048: Lanczos steps; tol: relative residual bound on the nev Ritz
 *   pairs; evals_host: K x nev double (host, ascending; NaN where fewer Ritz
 *   values exist); evec0_dev: NULL or K x dim double (device), the normalised
 *   lowest Ritz vector of each set.
 * The matrix-vector products are those of cih_ham_spmv (each stored nonzero
 * read once per product, FP32-pair arithmetic, fixed-point mirror sums),
 * with the bound taken as F (the Lanczos vectors have unit norm); the
 * orthogonalisation and the vectors stay FP64.
 * Library-allocated for the call: (max_iter + 2) x dim x K double of Lanczos
 * vectors and product scratch, dim x K int64 of mirror accumulators, and for
 * K > 1 an element-major copy of the values (K x nnz float).  Deterministic:
 * the same inputs give the same bits.  Returns 0, or 1 if some set did not
 * meet tol within max_iter (results still written), or a CIH_ERR_* code. */
int cih_lanczos_lowest(cih_basis_h h, const int64_t *rowptr_dev, const int32_t *col_dev,
                       const float *val_dev, int32_t K, int32_t nev, int32_t max_iter,
                       double tol, double *evals_host, double *evec0_dev, void *stream);

/* As cih_lanczos_lowest with the values element-major (val_em_dev[e * K + k],
 * the output of cih_ham_fill_batched), which the matrix-vector products read
 * directly: no element-major copy is made. */
int cih_lanczos_lowest_em(cih_basis_h h, const int64_t *rowptr_dev, const int32_t *col_dev,
                          const float *val_em_dev, int32_t K, int32_t nev, int32_t max_iter,
                          double tol, double *evals_host, double *evec0_dev, void *stream);

/* y = H x for K matrices sharing one structure, from the stored upper half
 * (the Lanczos product, Sec. 2): y_i = sum_{j >= i} h_ij x_j + sum_{j < i}
 * h_ji x_j, each stored nonzero read once.  The GPU's FP64 units are few, so
 * no FP64 operation runs per nonzero: x is split once into FP32 pairs
 * hi + lo, a product h (hi + lo) is formed as an FP32 pair (relative error
 * about 2^-47), and the row part is a double-float sum in an order fixed by
 * the structure.  Each strictly-upper h_ij x_i goes to column j's
 * accumulator as a 64-bit fixed-point integer (units 2^-s) by atomic adds,
 * which commute: the result is deterministic.  The scale keeps every
 * accumulator below 2^60 through the Cauchy-Schwarz bound
 * |sum_{i<j} h_ij x_i| <= F ||x||, F the Frobenius norm of the strictly-upper
 * values of all K sets and ||x|| the largest of the K vector norms; each
 * mirrored product is rounded to at most one unit 2^-s, about 2^-60 F ||x||.
 *   val_dev: K x nnz float (set-major) or, when values_em == 1, nnz x K
 *   (element-major, cih_ham_fill_batched's layout); x_dev, y_dev: dim x K
 *   double, element-major (x[i * K + s]), distinct arrays; 1 <= K <= 256.
 * Library-allocated for the call: dim x K int64 accumulators and FP32 pairs,
 * and for K > 1 set-major values an element-major copy (K x nnz float).  Stream-ordered;
 * synchronises only to read nnz when that copy is made.  An empty basis
 * (dim = 0) returns 0 at once, whatever the pointers.  Errors:
 * CIH_ERR_ARG, CIH_ERR_NOMEM, CIH_ERR_UNSUPPORTED (dim above 2^31),
 * CIH_ERR_CUDA. */
int cih_ham_spmv(cih_basis_h h, const int64_t *rowptr_dev, const int32_t *col_dev, const float *val_dev,
                 int32_t K, int32_t values_em, const double *x_dev, double *y_dev, void *stream);

/* Lanczos over row shards held by several processes (the paper distributes
 * the matrix over processes in chunks of equal nonzero count, Sec. 2 and 4.1;
 * cih_shard_rows and cih_ham_fill_rows build the shards).  Every process
 * calls this with its own rows [r0, r1) (col_dev / val_dev as cih_ham_fill_rows
 * wrote them, starting at stored nonzero rowptr[r0]) and the same other
 * arguments; the Lanczos vectors are replicated, so all processes compute the
 * same steps.  Each product runs on the local rows only: their row part goes
 * to yx_dev in FP64 and the mirrored part to acc_dev in the fixed-point units
 * of cih_ham_spmv (the scale set by f2, the squared Frobenius norm of the
 * whole matrix's strictly-upper values: the sum of cih_ham_upper_sumsq over
 * the shards).  The library then synchronises `stream` and calls
 * combine(ctx), which must replace both buffers by their sums over all
 * processes (an all-reduce: integer sums, and FP64 sums in which each entry
 * has one nonzero term, so both exact) and return 0.  The result is the same
 * on every process and, given the same scale, bit-identical to
 * cih_lanczos_lowest on the whole matrix.
 *   acc_dev: dim x K int64, yx_dev: dim x K double, both caller-owned and
 *   zero on entry (zero again on return); other arguments as
 *   cih_lanczos_lowest, values_em as cih_ham_spmv.
 * Errors: as cih_lanczos_lowest; a nonzero return of combine gives
 * CIH_ERR_ARG. */
int cih_lanczos_lowest_shard(cih_basis_h h, const int64_t *rowptr_dev, int64_t r0, int64_t r1, const int32_t *col_dev,
                             const float *val_dev, int32_t K, int32_t values_em, int32_t nev, int32_t max_iter,
                             double tol, double f2, uint64_t *acc_dev, double *yx_dev, int (*combine)(void *),
                             void *ctx, double *evals_host, double *evec0_dev, void *stream);

/* One shard's part of the bound cih_lanczos_lowest_shard needs: the sum of
 * the squares of the strictly-upper values (all K sets) of rows [r0, r1),
 * val_dev starting at stored nonzero rowptr[r0] (set-major K x nnz_shard, or
 * element-major when values_em == 1), into *f2_host.  Synchronises `stream`.
 * Errors: CIH_ERR_ARG, CIH_ERR_NOMEM, CIH_ERR_CUDA. */
int cih_ham_upper_sumsq(cih_basis_h h, const int64_t *rowptr_dev, int64_t r0, int64_t r1, const float *val_dev,
                        int32_t K, int32_t values_em, double *f2_host, void *stream);

/* Adjoint: d E0 / d t for every two-body table entry t of each of K sets,
 * given the normalised lowest eigenvectors psi (Hellmann-Feynman, E0 =
 * psi^T H psi): g_t = sum over stored (i, j) whose value uses t with sign s of
 * w * s * psi_i * psi_j, w = 2 off the diagonal and 1 on it.  Integer
 * arithmetic throughout, so the sum is deterministic: psi is held as
 * psi_i * 2^61 (int64), each product psi_i psi_j as the high word of the
 * 128-bit product (2^-58 units), and g accumulates in 2^-56 units.
 *   psi_dev: K x dim double (device), each set normalised: |psi_i| < 4
 *   and sum_i psi_i^2 <= 1 + 1e-6 (a larger entry counts as 0; either
 *   violation sets the device status that cih_check reports, since the
 *   fixed-point sums hold |g_t| < 128 and |g_t| <= 2 ||psi||^2); grad_dev: K x tbme_len double (device, caller-owned,
 *   overwritten).
 * Scratch: K x tbme_len int64 and K x dim int64, library-allocated for the
 * call.  Errors: CIH_ERR_ARG, CIH_ERR_NOMEM, CIH_ERR_CUDA. */
int cih_ham_tbme_grad(cih_basis_h h, const int64_t *rowptr_dev, int32_t K,
                      const double *psi_dev, double *grad_dev, void *stream);

/* One instance of a batch for cih_batch_solve: a basis with its own K
 * two-body tables.  Instances of one batch may differ in size, particle
 * numbers and Nmax. */
typedef struct {
    cih_basis_h basis;        /* in: from cih_basis_enumerate */
    int32_t K;                /* in: interaction sets of this instance, >= 1 */
    const float *tbme_dev;    /* in: K x tbme_len float, set-major (device) */
    const double *e_sp_dev;   /* in: NULL (HO energies) or n_orb_p + n_orb_n double (device) */
    double *evals_host;       /* out: K x nev double (host), ascending */
    double *grad_dev;         /* out: NULL, or K x tbme_len double (device): d E0 / d t */
    int64_t nnz;              /* out: stored nonzeros, from the count pass */
    int64_t bytes;            /* out: device bytes the instance holds while it is solved */
    int32_t wave;             /* out: admission wave it ran in, -1 if not admitted */
    int32_t status;           /* out: 0 converged, 1 not converged within max_iter,
                                 CIH_ERR_CAPACITY alone above the budget, or another CIH_ERR_* */
} cih_instance_t;

/* Fused build + Lanczos + adjoint for a batch of instances (Sec. 4.1's
 * count-then-compute passes, Sec. 2's Lanczos, and the Hellmann-Feynman
 * adjoint of cih_ham_tbme_grad), with admission by device memory:
 *   1. every instance's count pass and row-pointer scan (one concurrent
 *      branch per instance), then its nonzero count nnz;
 *   2. from nnz, each instance's bytes: rowptr, col, K x nnz values and the
 *      lowest Ritz vectors (held for the wave), plus the Lanczos and adjoint
 *      scratch (held one instance at a time);
 *   3. instances are admitted in the given order into waves whose peak stays
 *      within hbm_budget bytes (0 = 90% of the free device memory at the
 *      call); an instance above the budget on its own gets CIH_ERR_CAPACITY
 *      and is skipped;
 *   4. per wave: the fills of all its instances as one CUDA graph launch
 *      (one branch per instance), then per instance the lowest nev
 *      eigenvalues by Lanczos (as cih_lanczos_lowest with max_iter, tol) and,
 *      when grad_dev is given, d E0 / d t by the adjoint of the lowest Ritz
 *      vector; the wave's memory is released before the next wave.
 * All device memory is library-allocated for the call, except the caller's
 * tables and gradients.  Synchronises `stream`.  Returns 0 if every instance
 * has status 0, 1 if some instance has another status (see inst[i].status),
 * or a CIH_ERR_* code for the call itself (bad arguments, CUDA failure). */
int cih_batch_solve(cih_instance_t *inst, int32_t n, double hbar_omega, int32_t nev, int32_t max_iter,
                    double tol, int64_t hbm_budget, void *stream);

/* Synchronise `stream`, read and clear the basis' device error word.
 * Returns CIH_ERR_DEVICE if a kernel met a pair outside the table layout
 * (which the walk never produces for a consistent basis), else 0. */
int cih_check(cih_basis_h h, void *stream);

/* Eigen-decomposition of the symmetric tridiagonal matrix with diagonal
 * diag[n] and off-diagonal offdiag[n-1] (host arrays; offdiag may be NULL
 * when n = 1), the host step of cih_lanczos_lowest: implicit QR with
 * Wilkinson shifts.  evals[n] ascending; evecs (NULL or n x n, row-major)
 * holds eigenvector k in column k.  Errors: CIH_ERR_ARG, CIH_ERR_NOMEM. */
int cih_tridiag_eigen(int32_t n, const double *diag, const double *offdiag, double *evals, double *evecs);

/* Row-pointer scan that makes no device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate GPU
 * memory -- for example code that must run inside a framework whose memory
 * is all held by that framework's own pool, or a serving path that has
 * reserved its memory up front and may not call cudaMalloc (which can also
 * block the whole device) once it is running.
 *
 * Writes the exclusive prefix sum of counts_dev[0..n) into rowptr_dev[0..n]
 * (rowptr[0] = 0, rowptr[n] = total), the same result as the scan inside
 * cih_ham_count.  Both arrays are device memory owned by the caller;
 * counts_dev may equal rowptr_dev (scan in place), but the two must not
 * otherwise overlap (CIH_ERR_ARG).  Stream-ordered on `stream`; does not
 * synchronise.
 *
 * Scratch: the block sums live in a fixed 128 KiB array inside the library
 * (16,384 int64), which every GPU that loads the library holds until the
 * process exits.  Hence n is limited to 67,108,864 (16,384 tiles of 4,096
 * rows); larger n returns CIH_ERR_CAPACITY.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  The address is
 * kept for the life of the process: resetting the device (cudaDeviceReset or
 * a primary-context reset) after that first call is not supported.  All calls share
 * the array: calls whose work can overlap on the GPU (other streams, other
 * host threads) race and must be serialised by the caller.
 * Errors: CIH_ERR_ARG, CIH_ERR_CAPACITY, CIH_ERR_CUDA. */
int cih_rowptr_scan_static(const int64_t *counts_dev, int64_t n, int64_t *rowptr_dev, void *stream);

/* Number of kernels this library has launched in the process so far (all
 * devices, all handles): the difference across a region counts the region's
 * launches.  Errors: CIH_ERR_ARG. */
int cih_kernel_launches(int64_t *out);

const char *cih_strerror(int code);
const char *cih_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* CIH_H */

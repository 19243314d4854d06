/*
 * libdmrg -- C-ABI of the GB300 two-site DMRG hot path for nuclear shell-model
 * Hamiltonians (Legeza, Veis, Poves, Dukelsky, "Advanced density matrix renormalization
 * group method for nuclear structure calculations").
 *
 * Conventions common to every entry point
 * ---------------------------------------
 * - Every function returns an int status: DMRG_OK (0) or a negative DMRG_E* code.  No
 *   exception and no abort crosses the ABI; dmrg_last_error() returns a description of
 *   the last failure of a context (a pointer owned by the context, valid until the next
 *   call on it).
 * - Host arrays passed in are owned by the caller and copied before the call returns.
 * - Device buffers allocated by the library belong to the context and are released by
 *   dmrg_destroy().  Arguments documented as "device" are CUDA device pointers owned by
 *   the caller; they must hold the stated number of float64 elements.
 * - All work is issued on the stream given in dmrg_options.stream (NULL: the legacy
 *   default stream, which serialises with all other work on the device).  Calls that
 *   return numbers to the host synchronise that stream.  Contexts meant to run at the
 *   same time (the members of a batch) need streams of their own.
 * - Sectors are q = (N_p, N_n, 2M_z) integer triples in lexicographic order.  Chain
 *   position c holds site order[c]; bond b lies between positions b and b+1.
 * - A two-site step at position p (1 <= p <= N-3) treats the superblock
 *   (left block, positions 0..p-1) (x) site p (x) site p+1 (x) (right block, p+2..N-1)
 *   (two-site variant, "Xi_l (x) Lambda_{i+1} (x) Lambda_{i+2} (x) Xi_r").
 *   The wave function is block-sparse: one dense row-major block per enlarged-left sector
 *   Q_L whose partner q_T - Q_L exists on the enlarged right, blocks in Q_L order.
 */
#ifndef LIBDMRG_DMRG_H
#define LIBDMRG_DMRG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DMRG_OK 0
#define DMRG_EINVAL (-1)    /* bad argument, inconsistent input, or call out of order */
#define DMRG_ENOMEM (-2)    /* device or host allocation failed                       */
#define DMRG_ECUDA (-3)     /* a CUDA call failed (message has the CUDA error string)  */
#define DMRG_ENOCONV (-4)   /* an iteration stopped at its limit (Davidson, Jacobi SVD) */
#define DMRG_ETIMEOUT (-5)  /* a device-side wait gave up (bounded spin)               */

#define DMRG_FP64 0         /* every contraction in FP64                               */
#define DMRG_MIXED_FP32 1   /* operator contractions in FP32, Davidson/eig/energy FP64 */

#define DMRG_PRECOND_DIAG 0 /* Davidson correction r_i / (theta - D_i)                  */
#define DMRG_PRECOND_MLP 1  /* learned correction (falls back to DIAG until trained)    */

typedef struct dmrg_ctx dmrg_ctx;

/* The shell-model Hamiltonian of Eq. (1) on m-scheme orbitals alpha = (n,l,j,m,tau_z):
 *   H = sum_i eps_i n_i + sum_{i<j, k<l} vbar[ij,kl] c+_i c+_j c_l c_k
 * (antisymmetrised two-body matrix elements; the list must contain both (ij,kl) and
 * (kl,ij) and every entry must conserve N_p, N_n and 2M).  Indices are site indices. */
typedef struct {
  int32_t n_sites;          /* N, 4 <= N <= 64                                        */
  const int8_t* species;    /* [N] 0 = proton, 1 = neutron                             */
  const int8_t* two_m;      /* [N] 2 m of the orbital                                  */
  const double* eps;        /* [N] single-particle energies (MeV)                      */
  int64_t n_v;              /* number of two-body entries                              */
  const int32_t* v_idx;     /* [4 n_v] (i, j, k, l) with i < j and k < l               */
  const double* v_val;      /* [n_v] vbar (MeV)                                        */
  const int32_t* order;     /* [N] chain position -> site (a permutation)              */
  int32_t Np, Nn, two_Mz;   /* target sector ("m-scheme for J_z = 0": two_Mz = 0)      */
} dmrg_problem;

typedef struct {
  int32_t precision;        /* DMRG_FP64 or DMRG_MIXED_FP32                            */
  int32_t precond;          /* preconditioner: DMRG_PRECOND_DIAG or DMRG_PRECOND_MLP   */
  double dav_tol;           /* Davidson residual-norm tolerance (MeV), e.g. 1e-8       */
  int32_t dav_max_iter;     /* maximum H_eff products per step, e.g. 100               */
  int32_t dav_max_sub;      /* subspace size before thick restart, 4..64, e.g. 24      */
  void* stream;             /* cudaStream_t, NULL = default stream                     */
} dmrg_options;

/* Starting state: right-block bases for bonds b = N-3 down to 2.  The right block of
 * bond b is a truncation of (site b+1) (x) (right block of bond b+1); an enlarged sector
 * lists its rows piece by piece, site state 0 (block sector Q) then site state 1 (block
 * sector Q - q_site), each piece in block-state order.  For every kept sector: (N_p,
 * N_n, 2M, D, m) with D the enlarged dimension (must match) and a D x m row-major matrix
 * with orthonormal columns.  Replaces the paper's CI-DEAS warm-up. */
typedef struct {
  int32_t n_bonds;
  const int32_t* bonds;     /* [n_bonds] N-3, N-4, ..., 2                              */
  const int32_t* bond_ptr;  /* [n_bonds + 1] sector ranges                             */
  const int32_t* sec;       /* [5 n_sec] Np, Nn, 2M, D, m                              */
  const int64_t* u_off;     /* [n_sec + 1] element offsets into u                      */
  const double* u;          /* isometries                                              */
} dmrg_mps_init;

typedef struct {
  int32_t n_products;       /* H_eff applications                                      */
  int32_t converged;        /* 1 if residual <= dav_tol                                */
  double residual;          /* |H x - theta x|                                         */
  double energy;            /* Ritz value (MeV); FP64 Rayleigh quotient in mixed mode  */
  double heff_flops;        /* algorithmic flops of one H_eff product                  */
  double heff_bytes;        /* algorithmic bytes of one H_eff product                  */
  double seconds;           /* wall time of the call                                   */
  double energy1;           /* second targeted state (dmrg_set_roots(ctx, 2)), else NaN */
} dmrg_dav_stats;

typedef struct {
  int32_t p, dir;           /* position and direction (0 = left to right, 1 = back)    */
  int32_t n_products, kept;
  double energy, residual, trunc_err, seconds;
  double heff_seconds;      /* device time of the H_eff products (CUDA events)         */
  double heff_flops;        /* algorithmic flops of one H_eff product at this position */
  double heff_bytes;        /* algorithmic bytes of one H_eff product                  */
  double energy1;           /* second targeted state (dmrg_set_roots(ctx, 2)), else NaN */
} dmrg_step_stats;

/* Cumulative counters of a context since creation: kernel launches issued by the
 * library (all contexts of the process), H_eff products, their device time (CUDA events
 * on the context stream) and algorithmic flops and bytes, and the wall seconds spent in
 * the phases of the steps (host bookkeeping included). */
typedef struct {
  int64_t launches;
  int64_t heff_products;
  double heff_seconds;
  double heff_flops;
  double heff_bytes;
  double t_enlarge, t_super, t_davidson, t_truncate, t_project, t_predict;
  double t_sync;            /* host seconds blocked waiting for the context stream      */
  double t_enlarge_host;    /* host seconds of the enlargement's block discovery        */
  double t_upload;          /* host seconds inside table uploads (all contexts)         */
  int64_t upload_bytes;     /* bytes of those uploads (all contexts)                    */
  int64_t sb_blocks_l, sb_blocks_r, sb_terms, sb_tiles;   /* last superblock built (tiles:
                                                             32 x 32 tile kernels)       */
  /* finer host seconds: [0] superblock term lists, [1] product tiles, [2] tile validation
   * and uploads, [3] diagonal tasks, [4] renormalization tables, [5] renormalization
   * GEMMs (waited for), [6] operator index tables, [7] enlargement kernels (waited for),
   * [8] enlarged layouts, [9] source index uploads, [10] enlargement bitsets,
   * [11] enlargement block discovery, [12] enlarged block tables, [13] enlarged arena
   * allocation, [14] enlargement table uploads, [15] cudaMalloc calls (all contexts),
   * [16] Davidson: issuing the products, [17] Davidson: host work after each product,
   * [18] Davidson: waits after each product, [19] Davidson iterations (a count),
   * [20] truncation sectors too large for the cluster SVD, decomposed from the explicit
   * density matrix instead (a count), [21] truncations whose SVD stopped at its sweep
   * limit (a count), [22] H_eff products replayed from a CUDA graph (a count),
   * [23] reserved */
  double t_detail[24];
  int64_t pool_mallocs;     /* device allocations that missed the caching pool          */
  int64_t sb_small_tiles;   /* last superblock: tiles of the small-block product kernel */
  int64_t sb_term_hist[8];  /* last superblock: terms whose largest inner dimension is
                               <= 8, <= 16, <= 32, > 32 ([0..3]) and their flops ([4..7]) */
  double sb_kernel_flops;   /* last superblock: flops of one product in the association the
                               kernels use (psi R^T first), against the cheaper one counted
                               in heff_flops */
} dmrg_counters;

/* Create a context for one problem (Eq. 1 and a target state).  Validates the input
 * (permutation, index ranges, i<j and k<l, quantum-number conservation, Hermitian list)
 * and builds the normal / complementary operator partition on the host.  Status:
 * DMRG_EINVAL on invalid input, DMRG_ENOMEM.  The first call in a process sets glibc's
 * mmap threshold to 32 MB and its trim threshold to 1 GB (mallopt), so that the host
 * tables rebuilt at every step reuse heap memory instead of being paged in again. */
int dmrg_create(const dmrg_problem* prob, const dmrg_options* opt, dmrg_ctx** out);

/* Release every host and device resource of the context.  NULL is accepted. */
int dmrg_destroy(dmrg_ctx* ctx);

/* Description of the last error of the context (never NULL). */
const char* dmrg_last_error(const dmrg_ctx* ctx);

/* Build the block operators: the left block of bond 0 (site 0), the right block of bond
 * N-2 (site N-1), and the right blocks of bonds N-3..2 by renormalizing with the given
 * starting state (sweeping "from right to left" once).  Must precede every call below.
 * DMRG_EINVAL if the starting state does not match the sector structure. */
int dmrg_build_blocks(dmrg_ctx* ctx, const dmrg_mps_init* init);

/* Wave-function layout at position p.  Pass NULL arrays to query n_blocks and size;
 * then arrays of n_blocks entries: qn_left [3 n_blocks], dl, dr, off. */
int dmrg_psi_layout(dmrg_ctx* ctx, int32_t p, int64_t* n_blocks, int64_t* size,
                    int32_t* qn_left, int32_t* dl, int32_t* dr, int64_t* off);

/* psi_out = H_eff psi_in at position p with the current blocks (device pointers, size
 * from dmrg_psi_layout; in-place is not allowed).  The superblock Hamiltonian is
 * sum_k (L_k P^{|R_k|}) (x) R_k over the operator products of bond p (Section on the
 * two-site superblock).  Contractions in the context's precision. */
int dmrg_heff_apply(dmrg_ctx* ctx, int32_t p, const double* psi_in_dev, double* psi_out_dev);

/* Lowest eigenpair of H_eff at position p by Davidson's method (the variational
 * minimisation of the energy).  guess_dev: device vector (NULL = the context's
 * prediction from the previous step, or the uniform vector at the first step).
 * psi_out_dev: optional device copy of the normalised Ritz vector.  The eigenvector is
 * kept in the context for dmrg_truncate_renormalize.  DMRG_ENOCONV if the tolerance
 * was not reached within dav_max_iter products (energy and vector are still returned). */
int dmrg_davidson(dmrg_ctx* ctx, int32_t p, const double* guess_dev, double* psi_out_dev,
                  double* energy, dmrg_dav_stats* stats);

/* Truncation and renormalization after the Davidson step at position p (SVD theorem
 * basis change): dir 0 keeps M states of the enlarged left block (left block of bond p),
 * dir 1 of the enlarged right block (right block of bond p); reduced density matrix per
 * sector, FP64 eigendecomposition on the device, global selection of the M largest
 * weights (extended to the whole degenerate multiplet at the cut), and renormalization of
 * every normal and complementary operator of the new block.  trunc_err = discarded
 * weight; kept = number of kept states.  DMRG_EINVAL if no eigenvector is held for p;
 * DMRG_ENOCONV if a density-matrix decomposition stopped at its sweep limit (the
 * truncation and renormalization are still done). */
int dmrg_truncate_renormalize(dmrg_ctx* ctx, int32_t p, int32_t dir, int32_t M,
                              double* trunc_err, int32_t* kept);

/* One two-site step: H_eff at p, Davidson from the predicted guess, truncation and
 * renormalization in direction dir. */
int dmrg_step(dmrg_ctx* ctx, int32_t p, int32_t dir, int32_t M, dmrg_step_stats* st);

/* One sweep = positions 1..N-3 left to right then N-3..1 back ("sweeping back and
 * forth").  steps: optional array of 2(N-3) records.  energy: energy of the last step. */
int dmrg_sweep(dmrg_ctx* ctx, int32_t M, dmrg_step_stats* steps, double* energy);

/* Targeting of several states (the paper computes 2+ excitation energies by targeting the
 * two lowest eigenstates at once, so that their errors cancel in the difference).
 * n_roots = 1 (default) or 2.  With 2, every Davidson call seeks the two lowest
 * eigenpairs of H_eff (the lowest state whose residual is above dav_tol is corrected;
 * both must reach it), the truncation keeps the eigenvectors of the averaged reduced
 * density matrix (rho_0 + rho_1) / 2, and both wave functions are carried to the next
 * step by White's prediction.  The energies are returned in `energy` and `energy1` of
 * the statistics records.  Needs DMRG_FP64 and DMRG_PRECOND_DIAG (DMRG_EINVAL
 * otherwise, here and in dmrg_set_options while two states are targeted); not available
 * in batch mode; a superblock with fewer than two states fails with DMRG_EINVAL. */
int dmrg_set_roots(dmrg_ctx* ctx, int32_t n_roots);

/* Eigenvalues and eigenvectors of the reduced density matrix of the wave function held for
 * position p (after dmrg_davidson, dmrg_step or a sweep that ended at p), for every sector
 * of the enlarged block on side dir (0: left, the block the left-to-right truncation keeps
 * states of; 1: right) -- the decomposition behind the truncation's basis change by the
 * SVD theorem, computed by the same kernels (the singular vectors of each wave-function
 * block by one-sided Jacobi rotations, FP64); nothing is truncated or changed.  With two
 * targeted states the matrix is the average of the two.
 *   Call with NULL arrays to query n_sec and size (= sum of d^2); then qn [3 n_sec] (the
 * sectors, ascending), dims [n_sec], w [sum of d] (each sector's eigenvalues, descending,
 * clipped at 0), vecs [size] (optional: each sector's d x d row-major matrix whose columns
 * are the eigenvectors in the order of w, each with its largest |component| positive, the
 * lowest row on ties; the columns of zero eigenvalues may be zero).
 *   cluster: 0 = work split chosen per sector; 1, 8 or 16 = every sector whose shared-memory
 * share fits is decomposed by thread-block clusters of that many CTAs (the result is the
 * same up to rounding; this checks the partitioning).
 *   DMRG_EINVAL without a held wave function or for bad arguments; DMRG_ENOCONV if an SVD
 * stopped at its sweep limit (the results are still returned). */
int dmrg_rdm_eigh(dmrg_ctx* ctx, int32_t p, int32_t dir, int32_t cluster, int32_t* n_sec,
                  int64_t* size, int32_t* qn, int32_t* dims, double* w, double* vecs);

/* Orbital entropies of the two dots (the one-orbital entropy s_i = -Tr rho_i ln rho_i and
 * the two-orbital mutual information of the paper's entanglement analysis) from the
 * wave function held for position p (after dmrg_davidson, dmrg_step or a sweep that ended
 * at p; the lowest state when two are targeted), on the device.  rho: optional host array
 * of 16, the two-orbital reduced density
 * matrix of chain positions p and p+1, row-major, basis index 2 n_p + n_{p+1} (|00>,
 * |01>, |10>, |11>), rho[a][b] = sum_{l,r} psi(l,a,r) psi(l,b,r); it is diagonal except
 * for the |01>,|10> element, which equals <c+_{p+1} c_p> and is nonzero only when the two
 * orbitals have equal (species, m).  ent: optional host array of 4: s_p, s_{p+1}, the
 * two-orbital entropy s_{p,p+1} and the mutual information I = s_p + s_{p+1} - s_{p,p+1}
 * (natural logarithms; I >= 0, the paper prints the opposite sign convention).  A sweep
 * therefore gives s_i of every orbital at chain positions 1..N-2 and I of every
 * neighbouring pair.  DMRG_EINVAL if no wave function is held for p. */
int dmrg_dot_rdm(dmrg_ctx* ctx, int32_t p, double* rho, double* ent);

/* All-pairs orbital mutual information I_ij and one-orbital entropies s_i of the paper's
 * entanglement analysis (the quantities its orbital ordering is computed from), on the
 * device, from one left-to-right half sweep at M (positions 1..N-3, each as dmrg_step with
 * dir 0; the blocks and the held state change as in that half sweep).  The occupation and
 * the creation operator of every orbital of the growing left block are carried through the
 * renormalizations; the pair (i, j), i < j, is evaluated from the wave function of the
 * step where j is the left dot (j <= N-3), and the pairs with the last two chain positions
 * at the last step.  Each pair's two-orbital density matrix (basis |n_i n_j>, off-diagonal
 * <c+_i c_j>, nonzero only for equal species and m) gives s_i, s_j, s_ij and
 * I_ij = s_i + s_j - s_ij >= 0 (natural logarithms; the paper prints the opposite sign).
 * I: host array N x N, row-major, indexed by the problem's sites (not chain positions),
 * zero diagonal; s: host array N, from the last step's wave function; steps: optional host
 * array of N-3 step records.  DMRG_EINVAL before dmrg_build_blocks, for M < 1, NULL outputs
 * or two targeted states; DMRG_ENOCONV as dmrg_step (the results are still written). */
int dmrg_mutual_information(dmrg_ctx* ctx, int32_t M, double* I, double* s,
                            dmrg_step_stats* steps);

/* Dynamic block state selection (DBSS): the number of kept block states is set by the
 * truncation error instead of being fixed ("M_max determined by the truncation error
 * delta eps_TR" of the method section; the paper's runs use M_min = 256 and delta eps_TR =
 * 1e-3 ... 1e-6).  Once set, the M argument of dmrg_truncate_renormalize, dmrg_step,
 * dmrg_sweep and dmrg_batch_sweep is the ceiling M_max, and each truncation keeps
 *   - every state when the enlarged block has at most min(M_min, M_max) states;
 *   - otherwise the k largest weights (then the whole degenerate multiplet at the cut, as
 *     with a fixed M), k = the smallest count in [min(M_min, M_max), min(M_max, D)] whose
 *     discarded weight 1 - (lambda_1 + ... + lambda_k), summed in descending order in
 *     FP64, is at most trunc_target; k = min(M_max, D) if no count reaches it
 *     (D = dimension of the enlarged block).
 * trunc_target <= 0 switches back to a fixed M (the default).  DMRG_EINVAL if
 * trunc_target >= 1 or is NaN, or M_min < 1 with a positive target. */
int dmrg_set_dbss(dmrg_ctx* ctx, int32_t M_min, double trunc_target);

/* Orbital ordering from the two-orbital mutual information (host code, no context, no
 * device work): the paper orders the orbitals so that the entanglement distance
 * sum_ij I_ij |i - j|^2 is small, with spectral graph theory.  I: host n x n row-major
 * symmetric matrix of non-negative weights (the diagonal is ignored), 2 <= n <= 1024.
 * The graph Laplacian L = D - I is diagonalised (cyclic Jacobi, FP64); the eigenvector of
 * its second smallest eigenvalue (the Fiedler vector, normalised, sign such that the
 * lowest-index component within 1e-9 of the largest magnitude is positive) orders the
 * orbitals: order[k] = the orbital placed at chain position k, by ascending component,
 * equal components by index.  fiedler: optional host array of n for the vector.
 * DMRG_EINVAL for bad sizes, a non-finite, asymmetric or negative weight, or a
 * disconnected graph (second eigenvalue zero: no order between its parts).  When the
 * second and third eigenvalues coincide the order is not unique.  Thread-safe. */
int dmrg_fiedler_order(int32_t n, const double* I, int32_t* order, double* fiedler);

/* Extrapolation of energies in the number of kept block states (host code, no context,
 * no device work).  Points (M[i], E[i]), i < n, are fitted by ordinary least squares:
 *   DMRG_FIT_POWER:     E(M) = E_inf + X1 M^X2, the truncation-free estimate of the
 *                       method description; coef = {E_inf, X1, X2}, X2 sought in
 *                       [-8, -1e-4];
 *   DMRG_FIT_QUADRATIC: E = c0 + c1 / M + c2 / M^2, the second-order polynomial fit
 *                       that gives the upper bound in the 64Ge results (the paper does
 *                       not name the variable; 1/M here); coef = {c0, c1, c2}, c0 is the
 *                       estimate at M -> infinity.
 * rms = sqrt(mean squared residual).  coef: host array of 3; M, E: host arrays of n.
 * DMRG_EINVAL for fewer than three distinct M, M <= 0, a non-finite value, a NULL
 * pointer or an unknown kind; DMRG_ENOCONV when the best X2 lies on an end of its range
 * (the energies do not approach a limit as a power of M).  Thread-safe. */
#define DMRG_FIT_POWER 0
#define DMRG_FIT_QUADRATIC 1
int dmrg_extrapolate(int32_t kind, int32_t n, const double* M, const double* E, double* coef,
                     double* rms);

/* Sectors and dimensions of a stored block basis: side 0 = left block of bond b,
 * side 1 = right block of bond b.  NULL arrays query n. */
int dmrg_block_sectors(dmrg_ctx* ctx, int32_t side, int32_t b, int32_t* n, int32_t* qn,
                       int32_t* dims);

/* H_eff psi for callers that cannot allocate device memory during the call: processes
 * whose device memory is owned and budgeted up front by another allocator (for example a
 * serving framework that reserved the GPU), code that must not pay the implicit device
 * synchronisation of cudaMalloc / cudaFree, or code that cannot recover from a failed
 * allocation.  The paper has no counterpart; this is a service of the library.
 *   Result: the same product as dmrg_heff_apply, always with FP64 contractions.  Inputs
 * and outputs are the caller's device vectors as for dmrg_heff_apply.
 *   Storage: the intermediate of the two contraction stages lives in one file-scope
 * device array of 2,097,152 doubles (16 MiB) that every GPU loading the library holds
 * until the process exits.  No cudaMalloc, cudaFree or allocating library routine is
 * called.  A product that needs more intermediate storage is rejected with DMRG_EINVAL
 * and a message giving the size it needs.
 *   Preconditions: the superblock at p must already be set up by an allocating call at
 * the same position (dmrg_psi_layout or dmrg_heff_apply; they prepare this entry point's
 * task lists only for products that fit the array); otherwise DMRG_EINVAL.  The device the
 * context was created on must be current (DMRG_EINVAL otherwise): the array's address is
 * looked up on the current device.
 *   First call on a device: it looks up the array's device address (once per device,
 * with that device current; with lazy module loading the driver loads the code that
 * holds the array at that moment); make that first call before any stream capture.
 *   Concurrency: all calls share the one array.  Calls whose work overlaps on the GPU
 * (other streams, other contexts on the same device, other threads) race and corrupt
 * each other's results; serialise them. */
int dmrg_heff_apply_noalloc(dmrg_ctx* ctx, int32_t p, const double* psi_in_dev,
                            double* psi_out_dev);

/* Replace the options of a live context (precision, Davidson tolerances, stream); the
 * blocks are kept.  In DMRG_MIXED_FP32 the Davidson residual is computed from FP32
 * products, so the stopping test uses max(dav_tol, 1e-6 |theta|); the reported energy
 * is the FP64 Rayleigh quotient of the converged vector. */
int dmrg_set_options(dmrg_ctx* ctx, const dmrg_options* opt);

/* Learned Davidson preconditioner (not in the paper).  A network maps four features of
 * each wave-function element (asinh(theta - D_i), r_i and x_i normalised, the diagonal
 * correction normalised) through three ReLU layers of width 256 to the element of the
 * correction; it is trained on pairs that diagonal Davidson steps of this context
 * produce (target: the converged eigenvector's component orthogonal to the iterate) with
 * the library's own forward, backward and Adam kernels.  The preconditioner changes only
 * how the Davidson subspace grows, never the converged eigenpair.
 *   dmrg_mlp_reset: He-normal weights from a seed (SplitMix64), zero biases.
 *   dmrg_mlp_harvest: when enable != 0, every later Davidson run stores training pairs
 *     from its first eight iterates, per_iter elements each (fixed stride).
 *   dmrg_mlp_train: epochs of Adam over the harvested pairs, minibatch size batch;
 *     loss = mean squared error of the last epoch.  DMRG_EINVAL without samples.
 *   dmrg_mlp_params: dir 0 copies the parameters to host, dir 1 sets them (n must be
 *     dmrg_mlp_n_params()).  Packing: W1 (256x4), b1, W2 (256x256), b2, W3, b3, w4, b4.
 *   dmrg_mlp_loss_grad: loss and parameter gradient on given samples (B rows of 4
 *     features, B targets) in DMRG_FP64 or DMRG_MIXED_FP32 arithmetic (checks). */
int dmrg_mlp_reset(dmrg_ctx* ctx, uint64_t seed);
int dmrg_mlp_harvest(dmrg_ctx* ctx, int32_t enable, int32_t per_iter);
int dmrg_mlp_train(dmrg_ctx* ctx, int32_t epochs, int32_t batch, double lr, uint64_t seed,
                   double* loss, int64_t* n_samples);
int dmrg_mlp_params(dmrg_ctx* ctx, int32_t dir, double* host, int64_t n);
int dmrg_mlp_loss_grad(dmrg_ctx* ctx, int32_t precision, const double* params, const double* X,
                       const double* T, int64_t B, double* loss, double* grad);
int64_t dmrg_mlp_n_params(void);

/* Work split and launch mode of the kernels (not in the paper; results agree to rounding
 * whatever the split, and bit for bit whatever the launch mode, which the tests check).
 *   heff_big_edge: an output block of H_eff psi whose own dimensions or whose terms' input
 *     dimensions exceed this edge is computed by two grouped GEMM passes (T_k = psi R_k^T
 *     into a device scratch, then psi' = sum_k s_k L_k T_k; split-TF32 tensor cores in
 *     DMRG_MIXED_FP32, FP64 tiles in DMRG_FP64); smaller blocks by the fused tile kernels.
 *     0 = the fused kernels for every block; default 128 (measured on the headline
 *     workload at M = 4096: the grouped passes are as fast as the fused kernels on blocks
 *     of a few hundred states and 20x more accurate; on narrower blocks the fused kernels
 *     are faster).
 *   svd_cluster: thread-block cluster size of the truncation's SVDs: 0 = chosen per sector
 *     (default), or 1, 8 or 16 for every sector whose shared-memory share fits.
 *   heff_graph: 1 (default) = the kernels of the product that follow the staging of psi
 *     are captured as a CUDA graph at the second product of a precision on a superblock
 *     and replayed for every later product there (Davidson iterations, dmrg_heff_apply);
 *     0 = every kernel launched eagerly.  The FP64 energy of the mixed path (one product
 *     per step) is always eager.
 * Call between steps: the superblock held by the context is dropped and rebuilt at its next
 * use (a wave function held for truncation must be recomputed).  DMRG_EINVAL for values
 * out of range (heff_big_edge < 0 or > 4096, svd_cluster not 0, 1, 8 or 16, heff_graph not
 * 0 or 1). */
typedef struct {
  int32_t heff_big_edge;
  int32_t svd_cluster;
  int32_t heff_graph;
} dmrg_tuning;
int dmrg_set_tuning(dmrg_ctx* ctx, const dmrg_tuning* t);
int dmrg_get_tuning(dmrg_ctx* ctx, dmrg_tuning* t);

/* Autotuner of the product's work split (dmrg_tuning.heff_big_edge), on the superblock at
 * position p (not in the paper): one H_eff product is timed for each candidate edge (0 =
 * fused tile kernels only, then 32, 64, 128, 256) with CUDA events on the context stream,
 * best of reps >= 1 after two untimed products (the second captures the graph); the
 * fastest is kept, and within 5 % of it the smallest positive edge (its grouped passes sum
 * their products with compensation and are the more accurate).  The edge is set as by dmrg_set_tuning; the products agree to
 * rounding whichever is chosen, but the choice follows measured times.  chosen: the edge
 * set; edges, ms (optional host arrays of 5): the candidates and their best times.  Call
 * between steps (the superblock held by the context is dropped).  DMRG_EINVAL for a
 * position whose blocks are not available or reps < 1. */
int dmrg_autotune(dmrg_ctx* ctx, int32_t p, int32_t reps, int32_t* chosen, int32_t* edges,
                  double* ms);

/* Number of operator products L_k (x) R_k across bond b (0 <= b <= N-2) of the normal /
 * complementary operator partition built at dmrg_create: the terms the superblock
 * Hamiltonian sums over when the cut lies at bond b (labels that cannot connect the vacuum
 * to the full Hamiltonian are pruned).  Host data only, no device work.  DMRG_EINVAL for b
 * out of range. */
int dmrg_partition_terms(dmrg_ctx* ctx, int32_t b, int32_t* n_terms);

/* Read the cumulative counters. */
int dmrg_get_counters(dmrg_ctx* ctx, dmrg_counters* out);

/* Algorithmic cost of one H_eff product at position p: flops (2 per multiply-add, the
 * cheaper order of the two products of each term) and bytes (operator blocks read once
 * plus wave function in and out, at the element size of the context's precision). */
int dmrg_heff_cost(dmrg_ctx* ctx, int32_t p, double* flops, double* bytes, int64_t* n_items);

/* Batch mode (not in the paper; many independent problems at once).  A batch groups
 * contexts (1..64, same precision, blocks built).  dmrg_batch_sweep runs one sweep of
 * every context in lockstep: at step j each context does its own j-th two-site step
 * (position order as in dmrg_sweep; contexts with fewer steps drop out), and every
 * Davidson iteration computes the H_eff products of all contexts still iterating in ONE
 * fused kernel launch (tiles of all superblocks in one list), recorded once per step in a
 * CUDA graph on an internal stream and replayed with new vector pointers.  Each context's
 * own work (superblock, prediction, the host side of its Davidson iterations, truncation)
 * runs on a host thread of its own and on the context's stream, so contexts created with
 * distinct streams overlap.  Results are identical to sweeping the contexts one by one.
 * M: [n] kept states per context;
 * energies: optional [n] energy of each context's last step. */
typedef struct dmrg_batch dmrg_batch;
typedef struct {
  int64_t products;         /* batched product launches (graph replays included)        */
  double heff_seconds;      /* device time of those products (CUDA events)             */
  int64_t launches;         /* kernel launches issued by the library (graph nodes once) */
} dmrg_batch_stats;
int dmrg_batch_create(int32_t n, dmrg_ctx* const* ctx, dmrg_batch** out);
int dmrg_batch_destroy(dmrg_batch* b);
const char* dmrg_batch_last_error(const dmrg_batch* b);
int dmrg_batch_sweep(dmrg_batch* b, const int32_t* M, double* energies, dmrg_batch_stats* st);

#ifdef __cplusplus
}
#endif
#endif

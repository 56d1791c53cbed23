/*
 * hm.h -- C ABI of the GB300 sector Lanczos library (libhm.so).
 *
 * Implements the hot path of Schnack, Hage and Schmidt, "Optimized implementation of the
 * Lanczos method for magnetic systems" (arXiv:0706.3293): the matrix-free product
 * y = H x of the isotropic Heisenberg Hamiltonian, Eq. (E-2-1),
 *     H = - sum_b J_b s_{u_b} . s_{v_b},
 * restricted to one sector H(M) of fixed total magnetic quantum number (Sec. 3), in the
 * row-oriented form of Eq. (E-4-b) (Sec. 4), with the basis states numbered by the
 * paper's direct coding built on the dimension table D(N, A), Eq. (E-3-c), and the
 * decode/encode rules of Sec. 3.1 and 3.2; and the Lanczos recurrence built on it.
 *
 * Conventions shared by every entry point
 *   - Status: every function returns an int: HM_OK (0) on success, a positive
 *     informational code (HM_BREAKDOWN, HM_DEGENERATE) when the result is valid but
 *     noteworthy, a negative HM_E* code on error.  hm_last_error() returns a message for
 *     the last failing call of the calling host thread.  After HM_ECUDA the CUDA context
 *     may be unusable (a sticky device error).
 *   - Sites are numbered 0..n_sites-1.  A state is the digit string a_k = s - m_k in
 *     0..2s (Sec. 2); site k is digit position k, position n_sites-1 the most
 *     significant of the lexicographic order (Eq. E-3-a: a_1 varies fastest).
 *   - Sector: two_s = 2s (1..7), two_m = 2M; n_sites*two_s - two_m must be even and
 *     |M| <= N s.  The digit sum is A = N s - M.
 *   - Indices are 0-based (the paper's index minus one), dimension < 2^63.
 *   - Bonds: n_bonds entries (u[b], v[b], J[b]), 0 <= u, v < n_sites, u != v, at most
 *     HM_MAX_BONDS; each entry is one term -J_b s_u.s_v (a pair listed twice is summed).
 *     Bond arrays and all outputs documented "host" are host memory.
 *   - Vectors ("device") are caller-owned device memory on the current CUDA device,
 *     dense, row-major [dim][nvec], element type HM_F64 (double) or HM_F32 (float),
 *     aligned to the element size (16 bytes for nvec > 1).  Input and output vectors
 *     must not overlap.
 *   - stream is a cudaStream_t passed as void* (NULL: the legacy default stream).
 *     Calls without host results only enqueue work; calls with host results
 *     synchronise that stream before returning.
 *   - Workspace: functions that need scratch take a caller-owned device buffer
 *     (work, work_bytes); the matching *_workspace function gives the size.  The
 *     library allocates device memory only for small per-basis tables (in basis_build,
 *     and the block-path tables and run-time compiled kernels on the first call that
 *     needs them) and never frees caller memory; bond_corr_static allocates nothing.
 */
#ifndef HM_H
#define HM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    HM_OK = 0,
    HM_BREAKDOWN = 1,     /* Lanczos stopped early: beta_j below the breakdown threshold */
    HM_DEGENERATE = 2,    /* ground state (near-)degenerate: dE0/dJ is not unique       */
    HM_EINVAL = -1,       /* bad argument                                               */
    HM_EPARITY = -2,      /* N*2s - 2M odd, or |M| > N s                                */
    HM_EOVERFLOW = -3,    /* a dimension or table entry does not fit in 63 bits         */
    HM_ECUDA = -4,        /* a CUDA runtime call failed                                 */
    HM_ENOMEM = -5,       /* host allocation failed                                     */
    HM_ETIMEOUT = -6,     /* a device-side wait gave up (bounded spin) -- no hang       */
    HM_EWORKSPACE = -7    /* workspace missing or too small                             */
};

enum { HM_F64 = 0, HM_F32 = 1 };

#define HM_MAX_BONDS 512
#define HM_MAX_SITES 64

typedef struct hm_basis hm_basis;      /* library-owned: tables of one sector      */
typedef struct hm_lanczos hm_lanczos;  /* library-owned: state of one Lanczos run  */

/* Message of the last failing call on this host thread ("" if none). */
const char *hm_last_error(void);

/* ---- host-only helpers (no GPU needed) ---------------------------------------------- */

/* D(N, A) of Eq. (E-3-c) for the sector (n_sites, two_s, two_m): the number of basis
 * states of H(M) (Sec. 3).  HM_EPARITY / HM_EINVAL / HM_EOVERFLOW as above. */
int basis_dim_query(int n_sites, int two_s, int two_m, int64_t *dim);

/* Validates a bond list against n_sites (ranges, u != v, count, finite J). */
int bonds_check(int n_sites, int n_bonds, const int32_t *u, const int32_t *v, const double *J);

/* ---- basis (Sec. 3) ------------------------------------------------------------------- */

/* Builds D(k, a) by Eq. (E-3-c) and the per-position rank tables
 * CD[p][S][a] = sum_{n<a} D(p, S - n) (the inner sums of the Sec. 3.2 encoding) on the
 * host, and uploads them to the current device.  *out is library-owned; free it with
 * basis_free. */
int basis_build(int n_sites, int two_s, int two_m, hm_basis **out);

/* Spin-flip parity block of the s = 1/2 sector M = 0 (n_sites even, 10..32), a symmetry
 * reduction beyond the paper's sectors (its Sec. 1 names symmetries as the next way to
 * shrink a sector).  Flipping every spin (digit a -> 1 - a) maps the sector onto itself,
 * commutes with Eq. (E-2-1) and reverses the Sec. 3 order: index(flip w) = D - 1 -
 * index(w).  The basis keeps the representatives, the states with site N-1 up (digit
 * a_{N-1} = 0), which are indices 0 .. D/2 - 1 of the sector; a vector x on them stands for
 * the sector vector [x, parity * reversed(x)].  basis_dim gives D/2; basis_encode gives -1
 * for the other half.  matvec (one vector) and the Lanczos calls act as H restricted to
 * the block, through the s = 1/2 block kernels only (a bond list they cannot take fails
 * with HM_EINVAL); count_nnz, bond_corr and e0_grad return HM_EINVAL.  parity: +1 or -1. */
int basis_build_flip(int n_sites, int parity, hm_basis **out);
/* Momentum basis of a ring (translation symmetry; the paper names symmetries as a further
 * reduction of H(M) without constructing them): the sector (n_sites, two_s, two_m) split by
 * the cyclic translation T: site u -> u + 1 mod N, keeping the block of momentum k = 0 or,
 * for even N, k = N/2 (the real characters chi(n) = 1 and (-1)^n).  Basis states: one per
 * orbit of T whose period p has chi(p) = 1, |r^> = p^(-1/2) sum_{m<p} chi(m) T^m |r>, r the
 * orbit member with the smallest packed digit word, numbered in the order of the sector
 * index of r; basis_dim gives their number.  matvec, count_nnz, lanczos_*, arnoldi_run and
 * projection_run accept such a basis (one vector per product; the bonds must map onto
 * themselves under T with equal couplings, else HM_EINVAL); the other calls reject it.
 * Needs a sector of fewer than 2^32 states with N digits in 64 bits.  The device holds 8
 * bytes per sector state (a table from sector index to orbit, shift and period) plus 4 per
 * basis state.  HM_EINVAL for a bad k, or when no state has momentum k. */
int basis_build_momentum(int n_sites, int two_s, int two_m, int k, hm_basis **out);
int basis_free(hm_basis *basis);
int basis_dim(const hm_basis *basis, int64_t *dim);

/* Test hooks of the codec (Sec. 3.1 decode, Sec. 3.2 encode).  States are packed
 * digits: digit k in bits [k*b, k*b+b) of a uint64, b = 1 for 2s = 1, 2 for 2s <= 3,
 * 4 otherwise.  idx (device int64[n]) <-> states (device uint64[n]).  decode of an index
 * outside [0, dim) and encode of a state outside the sector give -1 / ~0ull. */
int basis_encode(const hm_basis *basis, const uint64_t *states, int64_t *idx, int64_t n,
                 void *stream);
int basis_decode(const hm_basis *basis, const int64_t *idx, uint64_t *states, int64_t n,
                 void *stream);

/* ---- the product y = H x: Eq. (E-4-b) ------------------------------------------------ */

/* y = H(J) x for nvec vectors at once (row-major [dim][nvec], 1 <= nvec <= 64).  Each
 * output row decodes its own index, applies every bond to its own state and gathers x
 * at the encoded targets (Sec. 4); rows never write each other's output.  dtype HM_F64
 * or HM_F32 for both x and y. */
int matvec(const hm_basis *basis, int n_bonds, const int32_t *u, const int32_t *v,
           const double *J, const void *x, void *y, int dtype, int nvec, void *stream);

/* Number of non-zero elements of H(M) for the bond list (one diagonal element per row plus
 * every allowed exchange; Sec. 4 counts of order N to N^2 of them per row), accumulated on
 * the device into *nnz (device int64, overwritten).  The figure behind Gnnz/s.  On a
 * momentum basis: the terms its product processes, one per row plus every allowed exchange
 * whose target orbit has a basis state. */
int count_nnz(const hm_basis *basis, int n_bonds, const int32_t *u, const int32_t *v, int64_t *nnz,
              void *stream);

/* Adjoint of the coupling dependence: out[b] = sum_i g_i [(s_u . s_v) x]_i for every
 * bond b (device double[n_bonds]), so that d(g^T H x)/dJ_b = -out[b] (H is linear in
 * J, Eq. E-2-1).  g, x: device vectors of dtype; nvec must be 1.  Deterministic:
 * fixed-order two-stage reduction in double.  work: bond_corr_workspace bytes. */
int bond_corr_workspace(const hm_basis *basis, int n_bonds, size_t *bytes);
int bond_corr(const hm_basis *basis, int n_bonds, const int32_t *u, const int32_t *v,
              const void *g, const void *x, double *out, int dtype, void *work,
              size_t work_bytes, void *stream);

/* bond_corr with no allocation and no workspace argument -- the paper has no counterpart.
 * For callers that cannot call cudaMalloc when they need the adjoint: a host program that
 * reserves its whole device-memory budget at start-up and forbids later allocation, or a
 * library embedded in a framework whose allocator owns all device memory.  The call
 * allocates nothing (no cudaMalloc, cudaFree or allocating library routine, on any call):
 * it runs the general row kernels, which read only the tables basis_build made, and keeps
 * their per-block partial sums in a file-scope device array of 1 MiB that every GPU
 * loading the library holds until exit.  A problem whose partial sums exceed it
 * (grid blocks x n_bonds doubles, at most 1216 x n_bonds on a 152-SM GPU) returns
 * HM_EINVAL with a message.  Output as bond_corr: out[b] (device double[n_bonds]), equal
 * to it up to the rounding of a different summation order.  The array is shared by all
 * calls and keeps the last call's contents (each call writes every slot it reads before
 * reading it); calls that overlap on the GPU race on it and must be ordered on one
 * stream.  The first call on a device (and the first after a new context is made there)
 * looks up the array's device address with cudaGetSymbolAddress; make that first call
 * before any stream capture. */
int bond_corr_static(const hm_basis *basis, int n_bonds, const int32_t *u, const int32_t *v,
                     const void *g, const void *x, double *out, int dtype, void *stream);

/* Seeded start vectors (device, dtype, nvec = 1).  kind 0: uniform on [-1, 1),
 * x_t = 2 (o_t >> 11) 2^-53 - 1; kind 1: +-1, x_t = -1 if bit 63 of o_t is set;
 * o_t = output t of SplitMix64 (Steele, Lea, Flood 2014) seeded with seed.  HM_F32
 * rounds the double value to nearest. */
int start_vector(const hm_basis *basis, uint64_t seed, int kind, void *x, int dtype,
                 void *stream);

/* ---- Lanczos --------------------------------------------------------------------------- */
/* Recurrence (three-term, Paige order, no re-orthogonalisation):
 *   v_1 = v0/|v0|;  u = H v_j - beta_{j-1} v_{j-1};  alpha_j = v_j . u;
 *   w = u - alpha_j v_j;  beta_j = |w|;  v_{j+1} = w / beta_j.
 * Breakdown after step j when beta_j <= tol * max(|alpha_1..alpha_j|,
 * beta_1..beta_{j-1}), tol = 1e-10 for HM_F64 vectors (the s = 1/2 and s = 1 block paths
 * update them in double-float arithmetic, unit roundoff about 2^-48, so a beta that is zero
 * in exact arithmetic comes out near 1e-12 of the scale) and 1e-5 for HM_F32 vectors (the
 * FP32 rounding floor); the run then stops with steps_done = j (status HM_BREAKDOWN).
 * Vectors are stored in dtype; alpha, beta and all reductions are double (fixed-order,
 * run-to-run deterministic); the tridiagonal eigensolve runs on the device in double. */

/* Workspace bytes of a Lanczos run with at most max_steps steps. */
int lanczos_workspace(const hm_basis *basis, int dtype, int max_steps, size_t *bytes);

/* Creates a run: copies the bonds, sets v_1 from v0 (device vector of dtype, or NULL
 * for the seeded uniform start vector), using caller workspace 'work'. */
int lanczos_init(const hm_basis *basis, int n_bonds, const int32_t *u, const int32_t *v,
                 const double *J, const void *v0, uint64_t seed, int dtype, int max_steps,
                 void *work, size_t work_bytes, void *stream, hm_lanczos **out);
/* Enqueues one fused step (matvec + alpha + update + beta) on stream; no host sync. */
int lanczos_step(hm_lanczos *run, void *stream);
/* One phase of a step: phase 0 = the product with its fused epilogue and alpha_j
 * (u = H v_j - beta_{j-1} v_{j-1}), phase 1 = the update and beta_j (w, v_{j+1}).
 * lanczos_step is phase 0 then phase 1; the split lets a caller time the product alone.
 * Phases must alternate starting with 0. */
int lanczos_substep(hm_lanczos *run, int phase, void *stream);
/* Copies alpha[0..steps_done), beta[0..steps_done) (host) and steps_done; syncs. */
int lanczos_read(hm_lanczos *run, double *alpha, double *beta, int *steps_done, void *stream);
int lanczos_free(hm_lanczos *run);
/* Name of the kernel that forms H q in each step of this run, NUL-terminated into
 * name[0..cap): "k_blk_lz64_jit" / "k_blk_lz32_jit" (s = 1/2 block product compiled for
 * this bond list at run time with NVRTC), "k_blk_lz64a_jit+k_blk_lz64b_jit" (the same FP64
 * product in two passes, for couplings in integer ratios, when the environment sets
 * HM_BLK_SPLIT=1: the bonds reaching site N-7 or above in a second pass that visits the
 * blocks with the top sites varying fastest; bit for bit the one-pass result), "k_blk_lz64" / "k_blk_lz32" (the same block
 * product reading its bonds from the parameters; used when NVRTC is unavailable or the
 * environment sets HM_JIT=0), "k_s1_lz64_jit" / "k_s1_lz32_jit" (s = 1 block product
 * compiled for the bond list), "k_s1_lz32" (its generic FP32 form) or "k_lz_matvec" (row
 * kernel of Eq. E-4-b for any s).  No counterpart in the paper: it reports an
 * implementation choice.  HM_EINVAL on NULL. */
int lanczos_kernel_name(const hm_lanczos *run, char *name, int cap);

/* Name of the kernel `matvec` launches for these arguments (the same dispatch; nothing
 * is launched, though a kernel specialised to the bonds may be compiled): "k_blk_matvec"
 * (s = 1/2 block kernel, up to 4 distinct couplings), "k_blk_matvec_jit" (block kernel
 * compiled at run time for a bond list with more distinct couplings), "k_s1_mv_jit" /
 * "k_s1_mv" (s = 1 block kernel compiled for the bond list / generic; FP32, one vector) or
 * "k_matvec" (general row kernel).  name: host buffer of cap bytes. */
int matvec_kernel_name(const hm_basis *basis, int n_bonds, const int32_t *u, const int32_t *v,
                       const double *J, int dtype, int nvec, char *name, int cap);

/* A whole run: steps steps captured in one CUDA graph and launched once, then the
 * n_ritz lowest eigenvalues of T (Sturm bisection on the device).  Host outputs:
 * alpha[steps], beta[steps], *steps_done, ritz[n_ritz].  Returns HM_OK or
 * HM_BREAKDOWN. */
int lanczos_run(const hm_basis *basis, int n_bonds, const int32_t *u, const int32_t *v,
                const double *J, const void *v0, uint64_t seed, int steps, int dtype,
                void *work, size_t work_bytes, double *alpha, double *beta,
                int *steps_done, double *ritz, int n_ritz, void *stream);

/* The lowest energy of every magnetisation sector: for A = 0 .. 2sN (sector 2M =
 * 2sN - 2A, i.e. M = Ns - A) one Lanczos run (lanczos_run) of up to `steps` steps from
 * the uniform start vector of seed sm64(seed, A * 2^20) (output #(A * 2^20) of SplitMix64;
 * the key the finite-temperature driver uses for the first vector of sector A), on the
 * sector coding of Sec. 3 and the products of Eq. (E-4-b).  e0[A] = the lowest Ritz value
 * of T (host, 2sN + 1 entries); steps_done[A] (host, may be NULL) = the run's length, less
 * than `steps` when the sector's Krylov space is exhausted (then e0[A] is exact).  The
 * paper has no routine of this name: its applications (Sec. 1) use this curve E0(M).
 * All 2sN + 1 runs are the branches of one CUDA graph, launched once on the stream: the
 * sectors are independent, so the small ones run side by side, and the lowest Ritz value of
 * each is found on the device (Sturm bisection).  work: device memory of
 * sector_ground_energies_workspace bytes (every sector's Lanczos workspace, back to back,
 * plus 24 bytes a sector of results), 256-byte aligned.  Synchronises the stream once, at
 * the end.  Errors as lanczos_run. */
int sector_ground_energies_workspace(int n_sites, int two_s, int steps, int dtype, size_t *bytes);
int sector_ground_energies(int n_sites, int two_s, int n_bonds, const int32_t *u, const int32_t *v,
                           const double *J, int steps, uint64_t seed, int dtype, void *work,
                           size_t work_bytes, double *e0, int *steps_done, void *stream);

/* Ground energy and its coupling gradient dE0/dJ_b = -<psi0| s_u.s_v |psi0>
 * (Hellmann-Feynman on Eq. E-2-1).  A first Lanczos pass gives T, its lowest
 * eigenvector c is found on the device (bisection + inverse iteration), a second pass
 * regenerates the same v_j and accumulates psi0 = sum_j c_j v_j, which is normalised;
 * then bond_corr(psi0, psi0).  Host outputs: *e0, dE0_dJ[n_bonds]; psi_out (device,
 * double[dim]) optional.  Returns HM_DEGENERATE when the gap to the second Ritz value of
 * that T is below 1e-8 |E0| (the gradient is then one of many).  One Krylov space holds
 * only one direction of an exactly degenerate eigenspace (the two dimer singlets of the
 * J2 = J1/2 ring), so such a degeneracy is not seen by one run: the result is then the
 * gradient at the ground state the start vector selects.  Workspace: e0_grad_workspace. */
int e0_grad_workspace(const hm_basis *basis, int n_bonds, int steps, size_t *bytes);
int e0_grad(const hm_basis *basis, int n_bonds, const int32_t *u, const int32_t *v,
            const double *J, const void *v0, uint64_t seed, int steps, void *work,
            size_t work_bytes, double *e0, double *dE0_dJ, double *psi_out, void *stream);

/* ---- Arnoldi and projection methods on the same product -------------------------------- */
/* The paper's closing summary ports its product to related Krylov-type methods such as
 * Arnoldi or the projection method without spelling them out; these are the textbook
 * iterations on the products of Eq. (E-4-b), FP64 vectors, no host round trip per step.
 *
 * Arnoldi with full re-orthogonalisation (classical Gram-Schmidt applied twice):
 *   v_1 = v0/|v0|;  for j = 1..steps: w = H v_j;  twice { h = V_j^T w; w -= V_j h;
 *   H[1..j, j] += h };  H[j+1, j] = |w|;  v_{j+1} = w / |w|.
 * V_j = (v_1 .. v_j) is kept in the workspace ((steps + 1) vectors).  The run stops after
 * step j when |w| <= 1e-12 * max |H entries| (Krylov space exhausted; HM_BREAKDOWN).
 * hess: host, (steps + 1) x steps doubles, column major (H[i, j] at hess[j (steps + 1) + i]),
 * may be NULL; *steps_done = columns formed; ritz: host, the n_ritz lowest eigenvalues of
 * the symmetric part of the leading steps_done x steps_done block (H is Hermitian, so in
 * exact arithmetic that block is the Lanczos tridiagonal matrix), NaN past steps_done.
 * v0: device double[dim] or NULL for the seeded uniform start vector (start_vector kind
 * 0).  Errors: HM_EINVAL (bad argument, zero start vector, spin-flip basis),
 * HM_EWORKSPACE, HM_ECUDA.  Synchronises the stream once at the end. */
int arnoldi_workspace(const hm_basis *basis, int steps, size_t *bytes);
int arnoldi_run(const hm_basis *basis, int n_bonds, const int32_t *u, const int32_t *v,
                const double *J, const void *v0, uint64_t seed, int steps, void *work,
                size_t work_bytes, double *hess, int *steps_done, double *ritz, int n_ritz,
                void *stream);

/* Projection (shifted power) method: psi_0 = v0/|v0|;  for k = 0..steps-1:
 *   y = H psi_k;  E_k = psi_k . y;  psi_{k+1} = (sigma psi_k - y) / |sigma psi_k - y|,
 * with |sigma psi_k - y|^2 = sigma^2 - 2 sigma E_k + y . y.  For sigma >= the largest
 * eigenvalue, psi_k tends to the ground state (largest eigenvalue of sigma - H) and E_k
 * decreases to E0.  sigma = 0 selects sum_b |J_b| s (s + 1), a bound on |E| of H.
 * energies: host double[steps] (E_0 .. E_{steps-1}); psi_out: device double[dim] or NULL,
 * receives psi_steps.  Errors as arnoldi_run.  Synchronises the stream once. */
int projection_workspace(const hm_basis *basis, int steps, size_t *bytes);
int projection_run(const hm_basis *basis, int n_bonds, const int32_t *u, const int32_t *v,
                   const double *J, const void *v0, uint64_t seed, int steps, double sigma,
                   void *work, size_t work_bytes, double *energies, double *psi_out,
                   void *stream);

/* Eigenvalues (ascending, host ev[n]) of the symmetric n x n host matrix a (row major; only
 * its symmetric part is used; not modified) by cyclic Jacobi rotations: the small dense
 * eigensolver arnoldi_run applies to its Hessenberg matrix.  No GPU involved.  HM_EINVAL
 * for NULL or n outside 1..4096. */
int sym_eigenvalues(int n, const double *a, double *ev);

/* ---- finite-temperature Lanczos over all sectors ---------------------------------------- */
/* Jaklic-Prelovsek estimator (cited by the paper, Sec. 1, as an application of the Lanczos
 * machinery) for s = 1/2 (two_s = 1), 10 <= n_sites <= 32, at most 4 distinct couplings and
 * 64 bonds.  Every sector A = N/2 - M (0..N) runs R (1..32) Lanczos runs of up to `steps`
 * steps from the +-1 vectors of SplitMix64 streams: stream seed = output #(A*2^20 + r) of
 * the generator seeded with `seed`, element t = -1 if bit 63 of output #t of that stream is
 * set, else +1.  Vectors are FP32 (row-major [rows][32], all sectors back to back),
 * reductions double-float then double; a run stops at beta_j <= 1e-5 * max(|alpha|, beta)
 * (above the FP32 noise floor).  A sector with D_A <= steps and D_A <= 512 would exhaust
 * its Krylov space, which FP32 vectors cannot detect: it is diagonalised exactly instead
 * (theta = its eigenvalues, tau = squared overlaps of the normalised start vector with the
 * eigenvectors, the limit the Lanczos quadrature reaches; its mlen = D_A).  Everything
 * runs in one CUDA graph: start vectors, one
 * cooperative persistent kernel for all steps (grid barriers wait at most 5 s, then the
 * call returns HM_ETIMEOUT), and the tridiagonal eigensolves on the device.  Outputs (host):
 * e_ref = lowest Ritz value; for each temperature T = temps[i]:
 *   Z[i] = sum_A (D_A/R) sum_r sum_j tau_j e^{-(theta_j - e_ref)/T}  (partition function
 *          divided by e^{-e_ref/T}),  E[i] = energy expectation;
 * optional theta/tau [(A*32 + r)*steps + j] and mlen [A*32 + r] (Krylov length).
 * vt: vectors per lane of the product (1, 2, 4), 0 = autotune (timed once per shape).
 * Returns the tiling used (> 0) or an error. */
int ftlm_workspace(int n_sites, int two_s, int n_bonds, const int32_t *u, const int32_t *v,
                   const double *J, int R, int steps, int n_t, size_t *bytes);
int ftlm_run(int n_sites, int two_s, int n_bonds, const int32_t *u, const int32_t *v,
             const double *J, int R, int steps, uint64_t seed, const double *temps, int n_t,
             double *Z, double *E, double *e_ref, double *theta, double *tau, int *mlen, int vt,
             void *work, size_t work_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HM_H */

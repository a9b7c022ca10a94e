/*
 * gbgreen.h — C ABI of the GB300 shifted Green's-function library.
 *
 * The library solves the generalized shifted linear equations
 *     (z_k S - H) x = b,   b = e_j,
 * for many complex energy shifts z_k (Im z_k > 0) and many unit right-hand
 * sides at once, with H a sparse real-symmetric tight-binding Hamiltonian and
 * S a sparse symmetric positive-definite overlap on the same pattern.  This is
 * the equation the order-N method of the paper is built on (Introduction:
 * generalized shifted linear equations used instead of the generalized
 * eigenproblem H y = lambda S y, cost order N).  The solutions are reduced on
 * the GPU to Green's-function outputs (local DOS, density-matrix and
 * energy-density elements on the sparsity pattern, local charge and energy).
 *
 * Solver: one seed Krylov space of A = S^{-1} H built by a conjugate
 * orthogonal CG (COCG) in the S-bilinear form, shared by every shift through
 * the collinear-residual recurrence.  S^{-1} is applied exactly by a
 * block-bidiagonal Cholesky factor of S where S's half-bandwidth is at most 63
 * (chains), else by an inner block-Jacobi-preconditioned iteration (CG, or
 * Chebyshev in the mixed path).  The paper defers the method's details to its
 * references; the recurrences used are the standard shifted COCG ones.
 *
 * Conventions for every entry point:
 *   - Return value: GB_OK (0) or a negative gb_status; gb_last_error() gives a
 *     thread-local message for the last failing call on the calling thread.
 *   - "host" pointers are read during the call only; "device" pointers are
 *     CUDA global-memory addresses on the current device, caller-owned.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     ordered on that stream.  Calls documented as synchronous wait for their
 *     own work before returning.
 *   - Device arrays must sit on their element's boundary (complex double 16
 *     bytes, double 8, float and int32 4); a misaligned array is GB_EINVAL.
 *   - The library never frees caller memory and never calls into PyTorch.
 */
#ifndef GBGREEN_H
#define GBGREEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GB_ABI_VERSION 2

typedef enum {
  GB_OK = 0,
  GB_EINVAL = -1,      /* invalid argument (shape, range, NULL, non-finite)   */
  GB_ENOMEM = -2,      /* device or host allocation failed / workspace small  */
  GB_ECUDA = -3,       /* a CUDA runtime call failed                          */
  GB_ENOTSPD = -4,     /* S not positive definite (diagonal block singular, or
                          the inner CG saw d^T S d <= 0)                      */
  GB_EBREAKDOWN = -5,  /* COCG breakdown (rho or gamma zero / non-finite) in at
                          least one column; its outputs are partial           */
  GB_ENOCONV = -6,     /* at least one (shift, column) pair did not reach tol
                          within maxit; all outputs are still written and
                          `converged` tells which pairs met tol              */
  GB_ETIMEOUT = -7     /* a bounded device wait (a staged factor tile of the
                          exact inner solve) gave up; outputs are unreliable */
} gb_status;

typedef enum {
  GB_FP64 = 0,  /* every vector, SpMM and reduction in FP64 */
  GB_MIXED = 1  /* reduced-precision vector work, FP64 scalars/recurrences */
} gb_precision;

/* Opaque matrix pair (H, S) resident on one device; library-owned. */
typedef struct gb_matrix gb_matrix;

typedef struct {
  int64_t n;          /* basis size (orbitals)                               */
  int64_t nnz;        /* scalar nonzeros of the shared CSR pattern            */
  int64_t nb;         /* block rows of the 4x4 BSR (n padded up to 4*nb)      */
  int64_t nnzb;       /* stored 4x4 blocks                                    */
  int32_t max_row;    /* longest pattern row (max |R_j|)                      */
  int32_t block;      /* block size (4)                                       */
  int32_t device;     /* CUDA device ordinal holding the matrix               */
  int32_t factor_bw;  /* S's half-bandwidth when the exact factor inner solve
                         is available (<= 63), else 0                        */
  double s_lam_min;   /* extreme eigenvalues of M^-1 S, M the 4x4 block       */
  double s_lam_max;   /* diagonal of S (Lanczos estimates at build time)      */
  int64_t factor_nblk; /* 64-row blocks of that factor (0: none)              */
} gb_matrix_info;

/*
 * gb_build_bsr — upload (H, S) and build the device block-sparse form.
 *
 * The operators of (z S - H) x = b (Introduction).  Input is one CSR pattern
 * shared by H and S, host memory, caller-owned:
 *   n        basis size, 1 <= n < 2^31
 *   row_ptr  [n+1] int64, row_ptr[0] = 0, non-decreasing
 *   col_idx  [nnz] int32, strictly increasing within each row, 0 <= c < n;
 *            the pattern must be symmetric and contain every diagonal entry
 *   h_val, s_val [nnz] float64, finite; both matrices must be symmetric
 * The CSR is regrouped on the host into 4x4 blocks over the orbital index
 * (blocks that hold no pattern entry are not stored; padding entries are
 * zero), copied to the device on `stream`, together with FP32 copies and the
 * inverses of S's 4x4 diagonal blocks (block-Jacobi preconditioner).
 * Returns GB_ENOTSPD if a diagonal block of S is not positive definite.
 * Synchronous.  On success *out owns device memory until gb_free(*out).
 */
gb_status gb_build_bsr(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                       const double* h_val, const double* s_val, void* stream,
                       gb_matrix** out);

/* gb_matrix_get_info — sizes of a built matrix (host struct, caller-owned). */
gb_status gb_matrix_get_info(const gb_matrix* m, gb_matrix_info* info);

/* gb_free — release a matrix (NULL is a no-op).  Synchronizes the device. */
void gb_free(gb_matrix* m);

/*
 * gb_block_factor_to_host — the factor of S that the exact inner solve uses,
 * computed on the host without a GPU (for inspection and tests).  S^{-1} is
 * applied once per Krylov iteration (the S-inner-product recurrence of the
 * shifted equations, Introduction); with half-bandwidth bw <= 63 the Cholesky
 * factor S = L L^T, cut into 64-row blocks (rows past n are identity), is
 * block lower bidiagonal with diagonal blocks D_i and sub-diagonal blocks C_i.
 * *bw receives S's half-bandwidth and *nblk the block count ceil(4 ceil(n/4)
 * / 64), or both 0 when bw exceeds 63 or S is not positive definite.
 * `factor` (host, caller-owned, may be NULL) receives 4 * nblk * 4096 doubles:
 * four arrays [nblk][64][64], each block stored k-major (entry (r, k) of the
 * block's matrix at k * 64 + r): D_i^-1, D_i^-T, E_i = D_i^-1 C_i and
 * F_i = D_i^-T C_{i+1}^T.  The solve is y_i = D_i^-1 f_i - E_i y_{i-1},
 * x_i = D_i^-T y_i - F_i x_{i+1}.
 */
gb_status gb_block_factor_to_host(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                  const double* h_val, const double* s_val, int32_t* bw, int64_t* nblk,
                                  double* factor);

/*
 * gb_bsr_to_host — the builder's block form, for inspection and tests.
 *
 * Runs the same host regrouping as gb_build_bsr without touching a GPU.
 * First call with all output pointers NULL to get *nb and *nnzb; then call
 * again with caller-owned host arrays:
 *   blk_ptr [nb+1] int32, blk_col [nnzb] int32,
 *   blk_h, blk_s [nnzb*16] float64 (row-major 4x4 per block).
 */
gb_status gb_bsr_to_host(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                         const double* h_val, const double* s_val, int64_t* nb,
                         int64_t* nnzb, int32_t* blk_ptr, int32_t* blk_col,
                         double* blk_h, double* blk_s);

/*
 * gb_spmm — Y = A X for A = H (which = 0) or S (which = 1).
 *
 * The sparse products of the Krylov recurrence for (z S - H) x = b
 * (Introduction: the order-N cost rests on sparse H and S; one product with H
 * per iteration, one with S per inner-iteration step).  X and Y are device arrays of n rows x w
 * complex columns, row-major with interleaved (re, im): element (i, c) at
 * [2*(i*w + c)] (re) and [2*(i*w + c) + 1] (im).  prec = GB_FP64: double
 * arrays and FP64 arithmetic; GB_MIXED: float arrays, FP32 arithmetic with
 * FP32 accumulation.  1 <= w <= 64.  Asynchronous on `stream`.
 */
gb_status gb_spmm(const gb_matrix* m, int32_t which, gb_precision prec, int32_t w,
                  const void* x, void* y, void* stream);

/*
 * gb_apply_sinv — Y = S^{-1} X with the exact block-bidiagonal Cholesky factor.
 *
 * The inner solve of the Krylov recurrence: the S-bilinear COCG applies S^{-1}
 * once per iteration to the product H p (the overlap S of the generalized
 * equations, Introduction).  On its own here, for tests and timing.  X and Y:
 * device arrays of n rows x w complex columns, layout as in gb_spmm;
 * prec = GB_FP64: double, one FP64 factor solve (exact to rounding);
 * GB_MIXED: float, one FP32 factor solve on TF32 tensor cores with a
 * three-term split (no refinement: ~2e-6 relative).
 * w in {1, 2, 4, 8, 16, 32}.  GB_EINVAL if the matrix has no factor (S's
 * half-bandwidth above 63).  Allocates its scratch on `stream` (stream-ordered
 * allocator) and frees it; synchronous.
 */
gb_status gb_apply_sinv(const gb_matrix* m, gb_precision prec, int32_t w, const void* x, void* y,
                        void* stream);

typedef struct {
  int32_t nshift;        /* K >= 1                                               */
  const double* z_re;    /* host [K] real parts of the shifts                   */
  const double* z_im;    /* host [K] imaginary parts, all > 0                   */
  const double* w_rho;   /* host [2K] complex weights c^rho_k (re, im pairs), or
                            NULL: rho / q / e_loc outputs are not formed       */
  const double* w_edm;   /* host [2K] complex weights c^E_k, or NULL            */
  int32_t nrhs;          /* number of right-hand sides e_j, >= 1                */
  const int32_t* rhs_cols; /* host [nrhs] orbital index j of each e_j            */
  double tol;            /* per-pair target ||b - (z S - H) x|| / ||b|| (> 0)    */
  int32_t maxit;         /* outer (seed) iteration cap (> 0)                     */
  gb_precision prec;     /* GB_FP64 or GB_MIXED                                  */
  double inner_tol;      /* iterative inner solve's relative residual; <= 0:
                            library default (FP64: 1e-14; mixed: 1e-7 per FP32
                            refinement level); unused by the exact factor solve */
  int32_t panel;         /* RHS columns per panel (1..32); <= 0: auto            */
  int32_t flags;         /* Inner solve S w = u.  Default: the exact
                            block-bidiagonal Cholesky solve where S's
                            half-bandwidth is <= 63 (FP64: one solve; mixed: two
                            FP32 solves around a float-float residual), else
                            an iteration (FP64: CG; mixed: Chebyshev).
                            bit 1: keep the inner-iteration vectors of a panel
                            in shared memory when they fit (iterations only);
                            bit 2: iterate with CG instead of the factor solve
                            (and instead of Chebyshev in the mixed path);
                            bit 4: mixed path iterates with Chebyshev instead
                            of the factor solve;
                            bit 5: mixed path forms H p as an unrefined FP32
                            product (faster, but its rounding makes the
                            recursive residual estimate drift below the true
                            residual: pair it with gb_true_residual);
                            bit 6: stop a column early once none of its open
                            shifts has halved its best residual in the last
                            3000 iterations (col_status 4 | 32; for use with
                            the correction solves, which set it themselves);
                            other bits are ignored                           */
  int32_t seed_shift;    /* index of the seed shift; < 0: middle of the grid     */
  int32_t reserved;
} gb_solve_params;

typedef struct {
  /* All device pointers, caller-owned; any may be NULL (that output is skipped). */
  double* ldos;       /* [K][nrhs]  -(1/pi) Im (G(z_k) S)_jj                        */
  double* rho;        /* [P] packed: for rhs c, entries off[c]..off[c+1]-1 hold
                         rho_ij = sum_k Im(c^rho_k G_ij(z_k)), i over the pattern
                         row j in increasing order; off = prefix sums of |R_j|   */
  double* edm;        /* [P] packed like rho, with the weights c^E_k            */
  double* q;          /* [nrhs] local charge  sum_i rho_ij S_ij                  */
  double* e_loc;      /* [nrhs] local energy  sum_i rho_ij H_ij                  */
  int32_t* iters;     /* [nrhs] seed iterations used                            */
  uint8_t* converged; /* [K][nrhs] 1 if the pair met tol                        */
  double* resid;      /* [K][nrhs] recursive residual estimate at exit          */
  double* g_proj;     /* [K][P][2] optional: G_ij(z_k) (re, im) on the pattern  */
  int32_t* inner_iters; /* [nrhs] inner steps of the column's panel summed over
                           the whole solve and all refinement levels: CG
                           iterations, Chebyshev steps, or one per level for
                           the exact factor solve                            */
  int32_t* col_status;  /* [nrhs] bit flags per column: 1 COCG breakdown, 2 S not
                           SPD, 4 a shift missed tol, 8 inner CG hit its cap,
                           16 a bounded wait for a factor tile gave up,
                           32 stopped early as stalled (flags bit 6)          */
} gb_outputs;

/*
 * gb_solve_workspace_size — bytes of device workspace gb_shifted_solve needs
 * for (m, p).  Returns 0 if the parameters are invalid (see gb_last_error).
 */
size_t gb_solve_workspace_size(const gb_matrix* m, const gb_solve_params* p);

/*
 * gb_solve_plan — the launch plan gb_shifted_solve would use for (m, p):
 * plan[0] = RHS columns per panel, plan[1] = teams (CTAs) launched,
 * plan[2] = 1 if the inner-iteration vectors live in shared memory,
 * plan[3] = dynamic shared-memory bytes per team, plan[4] = inner solve
 * (0 CG, 1 Chebyshev, 2 exact factor), plan[5] = teams resident per SM.
 * `plan` is a caller-owned host int32[6].
 */
gb_status gb_solve_plan(const gb_matrix* m, const gb_solve_params* p, int32_t* plan);

/*
 * gb_shifted_solve — solve (z_k S - H) x = e_j for every shift and RHS, and
 * reduce the solutions to the outputs in `out` (Introduction: generalized
 * shifted linear equations).
 *
 * `workspace` is caller-owned device memory of at least
 * gb_solve_workspace_size(m, p) bytes, 256-byte aligned; its contents on entry
 * are ignored.  One persistent launch processes every panel of RHS columns.
 * Synchronous: returns after the outputs are written.  GB_ENOCONV and
 * GB_EBREAKDOWN still write every output.
 */
gb_status gb_shifted_solve(const gb_matrix* m, const gb_solve_params* p, const gb_outputs* out,
                           void* workspace, size_t workspace_bytes, void* stream);

/*
 * gb_correct_unconverged — correction solve for the columns of a finished
 * gb_shifted_solve whose shifts missed tol (col_status bit 4; columns with a
 * breakdown or an indefinite S are left alone).  The paper's equation is the
 * same (Introduction); the correction is this library's answer to shifted
 * COCG's limited attainable accuracy: each such column is solved again alone,
 * in plain FP64 (exact factor inner solve where available), first with the
 * first solve's seed.  While shifts still miss tol, the worst remaining one
 * that has not been a seed yet seeds the next solve (six seeds at most), and
 * every shift keeps the result of the seed that served it best (its G_ij(z_k)
 * on the pattern row; rho, edm, q and e_loc are formed from those).  The
 * column's ldos, rho, edm, q, e_loc, iters and inner_iters (summed over the
 * seeds), converged, resid, g_proj and col_status entries in `out` are
 * overwritten.
 *
 * `p` and `out` are those of the first solve (out->col_status and out->resid
 * are required).  `workspace`: caller-owned device memory of at least
 * gb_correct_workspace_size(m, p, out->g_proj != NULL) bytes, 256-byte
 * aligned (one single-column solve plus its temporary outputs).  Synchronous.
 * `ncorrected` (host, may be NULL) receives the number of columns that now
 * meet tol.  Returns GB_OK when every re-solved column meets tol, GB_ENOCONV
 * if some still miss it (their outputs are then the FP64 solve's).
 */
gb_status gb_correct_unconverged(const gb_matrix* m, const gb_solve_params* p, const gb_outputs* out,
                                 void* workspace, size_t workspace_bytes, void* stream, int32_t* ncorrected);

/* Bytes of workspace gb_correct_unconverged needs (0: invalid parameters). */
size_t gb_correct_workspace_size(const gb_matrix* m, const gb_solve_params* p, int32_t want_g);

/*
 * gb_true_residual — FP64 true-residual check of a solve's columns.
 *
 * The shifted recurrence reports the recursive estimate ||rt_n|| / |pi^k_n|
 * of ||b - (z_k S - H) x^k|| (Introduction: the generalized shifted
 * equations); it equals the true residual only while every inner solve is
 * exact, so an inexact S^{-1} (an iterative inner solve, or reduced
 * precision) can report convergence that the true residual denies.  This call
 * re-runs the columns p->rhs_cols[ver[v]], v < nver, with the solve's own
 * parameters (same precision, seed, inner solve), keeping the history r_m on
 * every row, forms x^k = sum_m c^k_m r_m for every shift (a complex FP64
 * product of the history with the recurrence's coefficients) and evaluates
 * ||e_j - (z_k S - H) x^k||_2 in FP64 from the scalar CSR of H and S.
 *   nver        1..1024 columns to check (ver: host [nver], 0 <= ver[v] < nrhs)
 *   resid_true  device [K][nver] FP64 true residuals (caller-owned)
 *   out         NULL, or the outputs of the solve being checked: for every
 *               checked column whose true residual misses tol on some shift,
 *               col_status gets bit 4 and resid / converged take the true
 *               values, so gb_correct_unconverged re-solves it
 *   workspace   gb_true_residual_workspace_size(m, p, nver) bytes, 256-byte
 *               aligned: the history of every checked column, (maxit + 1) x
 *               4 ceil(n/4) x 16 bytes each, plus the solutions x^k
 *   nflagged    host, may be NULL: columns newly marked in `out`
 * Synchronous.  Costs one solve of the checked columns plus the product.
 */
gb_status gb_true_residual(const gb_matrix* m, const gb_solve_params* p, int32_t nver, const int32_t* ver,
                           double* resid_true, const gb_outputs* out, void* workspace, size_t workspace_bytes,
                           void* stream, int32_t* nflagged);

/* Bytes of workspace gb_true_residual needs (0: invalid parameters). */
size_t gb_true_residual_workspace_size(const gb_matrix* m, const gb_solve_params* p, int32_t nver);

/*
 * gb_fermi_density — chemical potential from the electron count, and the
 * Fermi-weighted density and energy-density matrices of a finished solve.
 *
 * The molecular dynamics of the paper needs the density matrix of the
 * occupied states at every step (Quantum molecular dynamics simulation); the
 * occupation needs the chemical potential mu, fixed by the electron count.
 * From a solve of EVERY orbital (p->nrhs = n, each orbital once) that kept
 * G_ij(z_k) (out.g_proj of gb_shifted_solve) and the local DOS, on an evenly
 * spaced real-axis grid z_k = eps_k + i eta (spacing d), with
 * f(x) = 1 / (1 + e^x) and spin degeneracy `spin`:
 *   c_k = -(spin / pi) f((eps_k - mu) / kT) d,   c^E_k = eps_k c_k,
 *   N(mu) = sum_j q_j = -pi sum_k c_k sum_j ldos[k][j]   (increasing in mu),
 * mu solves N(mu) = n_electrons (bisection to FP64 resolution), and
 *   rho_ij = sum_k c_k Im G_ij(z_k),  edm_ij = sum_k c^E_k Im G_ij(z_k),
 *   q_j = sum_i rho_ij S_ij,  e_loc_j = sum_i rho_ij H_ij,
 * all from the same solve (no second solve).
 *   g_proj, ldos  device outputs of that solve ([K][P][2], [K][nrhs])
 *   mu            host: the chemical potential
 *   out           its rho, edm, q, e_loc (device, caller-owned, any may be NULL
 *                 except that q / e_loc need rho) are overwritten
 *   workspace     gb_fermi_workspace_size(m, p) bytes, 256-byte aligned
 * GB_EINVAL if the shifts are not evenly spaced, or the electron count lies
 * outside what the grid holds.  Synchronous.
 */
gb_status gb_fermi_density(const gb_matrix* m, const gb_solve_params* p, const double* g_proj, const double* ldos,
                           double n_electrons, double kT, double spin, double* mu, const gb_outputs* out,
                           void* workspace, size_t workspace_bytes, void* stream);

/* Bytes of workspace gb_fermi_density needs (0: invalid arguments). */
size_t gb_fermi_workspace_size(const gb_matrix* m, const gb_solve_params* p);

/*
 * gb_forces — atomic forces from the density and energy-density matrices of a
 * finished solve of every orbital.
 *
 * The paper's molecular dynamics moves the atoms with forces from each step's
 * electronic structure (Quantum molecular dynamics simulation).  For a
 * non-orthogonal two-center tight-binding model at fixed chemical potential,
 *   F_a = -Tr[rho dH/dR_a] + Tr[P^E dS/dR_a],
 * with rho and P^E the solve's (or gb_fermi_density's) packed outputs; the
 * traces run over both orders of every element (rho_ij from column j and
 * rho_ji from column i), so they are exact for the matrices as computed.
 *   p          the solve's parameters: rhs_cols must hold every orbital once
 *   rho, edm   device [P], packed as gb_outputs.rho / edm of that solve
 *   grad_h, grad_s  device [3][nnz]: per element of the CSR given to
 *              gb_build_bsr (same order), the gradient of H_ij (S_ij) with
 *              respect to the position of the atom of orbital i (row); the
 *              gradient with respect to the other atom is its negative
 *              (two-center elements); entries within one atom are ignored
 *   atom_off   host [n_atoms + 1]: atom a owns orbitals atom_off[a] ..
 *              atom_off[a+1]-1 (consecutive), atom_off[0] = 0, atom_off[n_atoms] = n
 *   forces     device [n_atoms][3], overwritten
 *   workspace  gb_forces_workspace_size(m, p, n_atoms) bytes, 256-byte aligned
 * GB_EINVAL on a partial column set or bad atom ranges.  Synchronous.
 */
gb_status gb_forces(const gb_matrix* m, const gb_solve_params* p, const double* rho, const double* edm,
                    const double* grad_h, const double* grad_s, const int64_t* atom_off, int32_t n_atoms,
                    double* forces, void* workspace, size_t workspace_bytes, void* stream);

/* Bytes of workspace gb_forces needs (0: invalid arguments). */
size_t gb_forces_workspace_size(const gb_matrix* m, const gb_solve_params* p, int32_t n_atoms);

/*
 * gb_add_sinv_terms — the non-resolvent terms of a pole expansion of the Fermi
 * function, added to a finished solve's outputs.
 *
 * The paper leaves the choice of shifts open (Introduction).  Expanding the
 * Fermi function in poles w_p off the real axis, f(x) ~ 1/2 + sum_p R_p
 * [1/(x - i a_p) + c.c.] (x = (eps - mu)/kT), makes rho and P^E sums of
 * resolvents G(w_p), which the solve forms from weights c_k, plus
 *   rho += a_rho S^-1,    P^E += b_edm S^-1 + c_shs S^-1 H S^-1
 * on the pattern, which no resolvent gives.  This call adds those terms for
 * the solve's columns (FP64 factor solves; needs S's half-bandwidth <= 63) and
 * recomputes q and e_loc from the completed rho.
 *   p        the solve's parameters (its rhs_cols)
 *   out      its rho / edm are updated in place (either may be NULL), q and
 *            e_loc overwritten when present
 *   workspace gb_add_sinv_terms_workspace_size(m, p) bytes, 256-byte aligned
 * GB_EINVAL without a factor, GB_ETIMEOUT if a bounded wait of a factor pass
 * gave up.  Synchronous.
 */
gb_status gb_add_sinv_terms(const gb_matrix* m, const gb_solve_params* p, double a_rho, double b_edm, double c_shs,
                            const gb_outputs* out, void* workspace, size_t workspace_bytes, void* stream);

/* Bytes of workspace gb_add_sinv_terms needs (0: invalid arguments). */
size_t gb_add_sinv_terms_workspace_size(const gb_matrix* m, const gb_solve_params* p);

/*
 * gb_wavepacket — propagate wavepackets by i S dc/dt = H c.
 *
 * The transport simulations of the paper propagate a hole wavepacket with a
 * Schroedinger-type equation from an eigenstate such as the HOMO, with a step
 * of ~0.1 fs (Quantum wavepacket dynamics).  Each of `nsteps` steps applies
 * exp(-i tau S^-1 H) by its Chebyshev (Jacobi-Anger) series in
 * A~ = (S^-1 H - b) / a, b, a the centre and half-width of [e_min, e_max]:
 * one H product and one FP64 factor solve of S per term, the series cut where
 * |J_k(a tau)| < 1e-17.
 *   nwp       number of wavepackets (columns)
 *   psi       device complex double [n][nwp] (re, im), in/out
 *   tau       step in hbar / eV (0.1 fs = 0.15193 / eV)
 *   e_min, e_max  bounds that contain every generalized eigenvalue of (H, S):
 *             the series diverges outside them, so take them with a margin
 *   nterms_out (host, may be NULL) receives the series length per step
 *   workspace gb_wavepacket_workspace_size(m, nwp) bytes, 256-byte aligned
 * GB_EINVAL without a factor (S's half-bandwidth above 63) or if a step needs
 * more than 256 terms.  Synchronous.
 */
gb_status gb_wavepacket(const gb_matrix* m, int32_t nwp, void* psi, int32_t nsteps, double tau, double e_min,
                        double e_max, int32_t* nterms_out, void* workspace, size_t workspace_bytes, void* stream);

/* Bytes of workspace gb_wavepacket needs (0: invalid arguments). */
size_t gb_wavepacket_workspace_size(const gb_matrix* m, int32_t nwp);

/*
 * gb_shifted_solve_batched — many independent systems in one persistent launch.
 *
 * The shifted equations of the Introduction for many independent structures
 * at once (the Quantum molecular dynamics section solves one polymer bundle
 * per MD step; independent chains of uneven length are this entry point's
 * unit of work).  Each system s solves (z_k S_s - H_s) x = e_j for its own shifts and columns
 * (params[s]) on its own matrix mats[s] and writes its own outputs outs[s];
 * all systems share one precision and one device.  Work items are (system,
 * panel of `panel` columns) pairs taken from a device counter, largest systems
 * first; converged shifts and columns retire inside their panel.  panel <= 0:
 * library choice.  `workspace`: gb_batched_workspace_size bytes, 256-byte
 * aligned.  Synchronous; the status is the worst over all systems.
 */
gb_status gb_shifted_solve_batched(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                                   const gb_outputs* outs, int32_t panel, void* workspace,
                                   size_t workspace_bytes, void* stream);

/* Workspace bytes for gb_shifted_solve_batched (want_g: any system asks for g_proj). */
size_t gb_batched_workspace_size(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                                 int32_t panel, int32_t want_g);

/*
 * gb_correct_batched — the correction solve of a finished gb_shifted_solve_batched
 * (same systems, params and outputs).  Every column, of every system, whose
 * shifts missed tol (col_status bit 4, no breakdown, S definite) is solved again
 * in ONE batched launch: plain FP64, exact factor inner solve where available,
 * the first solve's seed, one column per panel.  The columns that then meet tol
 * replace their entries in `outs` (ldos, rho, edm, q, e_loc, iters,
 * inner_iters, converged, resid, g_proj, col_status).  Columns that still miss
 * tol go through gb_correct_unconverged (seed switching), system by system.
 *
 * `workspace`: gb_correct_batched_workspace_size(...) bytes for the same
 * arguments, 256-byte aligned.  Both calls read every system's col_status from
 * the device (they wait on `stream`).  `ncorrected` (host, may be NULL): columns
 * that now meet tol.  Returns GB_OK when every column meets tol, GB_ENOCONV if
 * some still miss it.  Synchronous.
 */
gb_status gb_correct_batched(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                             const gb_outputs* outs, void* workspace, size_t workspace_bytes, void* stream,
                             int32_t* ncorrected);

/* Bytes of workspace gb_correct_batched needs now (256 if no column failed; 0: invalid arguments). */
size_t gb_correct_batched_workspace_size(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                                         const gb_outputs* outs, void* stream);

/*
 * gb_tune_panel_batched — autotuner for the batched panel width: runs the
 * batch with every maxit capped at probe_maxit for panel widths {8, 16, 32},
 * times each launch on `stream`, and returns the fastest in *best_panel
 * (times_ms: optional host float[3], -1 for a width that did not fit the
 * workspace).  The outputs are overwritten by the probe runs.
 */
gb_status gb_tune_panel_batched(int32_t nsys, const gb_matrix* const* mats, const gb_solve_params* params,
                                const gb_outputs* outs, int32_t probe_maxit, void* workspace,
                                size_t workspace_bytes, void* stream, int32_t* best_panel, float* times_ms);

/*
 * gb_shifted_solve_static — gb_shifted_solve without any allocation.
 *
 * It solves the same generalized shifted equations (Introduction); the paper
 * has no counterpart for the memory scheme: this entry point exists for
 * callers that may not allocate once they run — an application whose device memory belongs to
 * another runtime's pool that already claims the whole GPU, or a
 * latency-critical loop where cudaMalloc's implicit device synchronisation is
 * not acceptable.  Same arguments and results as gb_shifted_solve (caller-owned
 * outputs), but the scratch is a fixed per-device array inside the library of
 * gb_static_scratch_bytes() bytes (32 MiB), which every GPU that loads the
 * library holds until the process exits; the launch header and status are
 * staged in fixed host buffers.  No cudaMalloc, cudaFree or other allocating
 * routine is called.
 *   - The first call on a device looks up the scratch's device address (once
 *     per device, with that device current).
 *   - Problems whose scratch exceeds the array, or with nrhs > 4096, are
 *     rejected (GB_ENOMEM / GB_EINVAL) with a message naming the limit; the
 *     number of concurrent teams is reduced when that lets the problem fit
 *     (results do not depend on it).
 *   - Every call shares the one array and leaves its contents behind; the call
 *     re-initialises everything it reads (the work counter is cleared from
 *     the host).  Calls whose GPU work overlaps (other streams, other host
 *     threads) race on the array: serialise them.
 * Synchronous: the call waits on `stream` for its own work (it reads the
 * per-column status back) before it returns.
 */
gb_status gb_shifted_solve_static(const gb_matrix* m, const gb_solve_params* p, const gb_outputs* out,
                                  void* stream);

/* Size in bytes of the per-device scratch of gb_shifted_solve_static. */
size_t gb_static_scratch_bytes(void);

/* Thread-local message describing the last error on this thread ("" if none). */
const char* gb_last_error(void);

/* GB_ABI_VERSION of the loaded library. */
int32_t gb_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GBGREEN_H */

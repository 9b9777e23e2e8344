/*
 * mrom.h -- C ABI of the GB300 reduced-order MPT spectral-signature library.
 *
 * The library computes magnetic polarizability tensor (MPT) spectral
 * signatures with the reduced-order "Matrix Method" of Elgy & Ledger,
 * "Efficient Computation of Magnetic Polarizability Tensor Spectral
 * Signatures for Object Characterisation in Metal Detection":
 *   snapshots D_i (Sect. 4.1, Eq. (13)) -> truncated SVD (Eqs. (14), (15))
 *   -> Galerkin projection of K and C (Eq. (17)) -> for many objects and
 *   frequencies the reduced solves (Eq. (17)) and the tensor post-processing
 *   R (Eq. (18)) and I (Eq. (19)) -> the a-posteriori certificate Delta
 *   (Lemma 4.2, Eq. (20)) -> adaptive snapshot selection (Algorithm 1).
 *
 * Conventions used throughout
 *  - Sign convention of the paper: A[omega] = K - i omega C + eps M, source
 *    r_i = i omega C o_i (Sect. 3.1, Eq. (9)).  A solution written for the
 *    conjugate convention (K + i omega C) alpha = i omega b is alpha = -conj(q).
 *  - Complex numbers are interleaved (re, im) float64 pairs (complex128,
 *    cuDoubleComplex); matrices are row-major.
 *  - Tensor outputs are float64 arrays [n_obj][n_w][3][3], row-major.
 *    R excludes N0 unless the object was given an N0 (then R~ = N0 + R).
 *  - Unless stated otherwise, array arguments of compute calls are DEVICE
 *    pointers owned by the caller; they must stay valid until the handle's
 *    stream has reached the call.  Object-creation calls accept host or
 *    device pointers (copied with cudaMemcpyDefault before returning).
 *  - Every compute call is asynchronous on the handle's CUDA stream.  A call
 *    returns MROM_EINVAL for invalid arguments (nothing is launched),
 *    MROM_ECUDA for a failed launch, MROM_ENOMEM when device memory runs out.
 *    Conditions detected on the device (a non-finite frequency, a zero or
 *    non-finite pivot) are recorded in a device status word and returned by
 *    the next mrom_synchronize() on the handle.  No call aborts the process.
 *  - No call is thread-safe on the same handle.
 */
#ifndef MROM_H
#define MROM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MROM_OK = 0,
  MROM_EINVAL = 1,        /* bad argument (shape, null pointer, non-finite value) */
  MROM_ENOMEM = 2,        /* device allocation failed */
  MROM_ECUDA = 3,         /* CUDA runtime error (launch, copy) */
  MROM_ESINGULAR = 4,     /* zero or non-finite pivot in a reduced solve */
  MROM_ENOTCONVERGED = 5, /* iteration limit reached */
  MROM_ETIMEOUT = 6,      /* a bounded device wait gave up */
  MROM_ECALLBACK = 7,     /* a user callback returned an error */
  MROM_ENOTSUP = 8        /* option not supported for this object */
} mrom_status;

typedef enum { MROM_FP64 = 0, MROM_MIXED = 1 } mrom_precision;
typedef enum { MROM_SOLVER_AUTO = 0, MROM_SOLVER_LU = 1 } mrom_solver;

typedef struct mrom_ctx* mrom_handle;
typedef struct mrom_rom* mrom_rom_t;
typedef struct mrom_plan_s* mrom_plan;

/* ---------------------------------------------------------------- context */

/* Create a handle on CUDA device `device`.  `cuda_stream` is the cudaStream_t
 * every call of this handle runs on (NULL: CUDA's default stream).  The
 * handle owns a small device status word and no other device memory.  The
 * library's per-call buffers are stream-ordered allocations from the device's
 * default memory pool; the first handle raises that pool's release threshold
 * (a setting of this process) to 8 GiB, so that freed buffers stay mapped for
 * the next call instead of returning to the driver at each synchronisation. */
mrom_status mrom_create(int device, void* cuda_stream, mrom_handle* out);
mrom_status mrom_destroy(mrom_handle h);
/* Replace the stream used by later calls (NULL: CUDA's default stream). */
mrom_status mrom_set_stream(mrom_handle h, void* cuda_stream);
/* Wait for the handle's stream; returns the first CUDA error or the first
 * device-detected condition since the previous mrom_synchronize, then clears it. */
mrom_status mrom_synchronize(mrom_handle h);
/* Human-readable description of the last error on this handle (never NULL). */
const char* mrom_last_error(mrom_handle h);
/* Number of kernels this library launched on the handle so far. */
int64_t mrom_launch_count(mrom_handle h);
/* Precision of mrom_project / mrom_project_dirs on this handle.  MROM_FP64
 * (default): every product in float64.  MROM_MIXED: the SpMM K U in complex64,
 * and the Gram products K_r, C_r, eps M_r and b on the tensor cores from complex64
 * operands (each real part split into two TF32 parts, three products accumulated in
 * FP32 over 128 rows at a time, the partials summed in float64); the TSVD and the
 * certificate Gram stay float64.  Requires r <= 112. */
mrom_status mrom_set_projection_precision(mrom_handle h, mrom_precision precision);

/* ------------------------------------------------------- reduced objects */

/* One reduced object with a single basis U (N x r) shared by the three
 * directions (Remark 3.1 taken one step further: one space for all i).
 * With this basis, Sect. 4.3 needs
 *   K   = U^H K U        r x r complex128, Hermitian     (K_ij^M, Eq. (18))
 *   C   = U^H C U        r x r complex128, Hermitian PD  (C_ij^M, Eq. (19))
 *   Me  = U^H (eps M) U  r x r or NULL (added to A only; Eq. (17))
 *   B   = [b_1 b_2 b_3]  r x 3 complex128, b_i = U^H C o_i, so that the
 *         reduced source is U^H r_i = i omega b_i and the o^T C^(2) U p and
 *         t^M p terms of Eq. (19) are b_i^H p_j
 *   c00 = o_i^T C^(1) o_j + c_ij + s_i^T o_j + s_j^T o_i   (3 x 3 float64)
 *   G   = Phi^H X^-1 Phi, (2r+3) x (2r+3) complex128 Hermitian, or NULL
 *         (then no certificate), with the columns of Phi ordered
 *         [C o_1, C o_2, C o_3 | (K + eps M) U | C U]  (Lemma 4.2)
 *   K_in (r x r or NULL): the part of K scaled by a permeability scale s_mu,
 *         K(s_mu) = (K - K_in) + K_in / s_mu.
 *   N0  (9 float64 or NULL): added to R (Eq. (6a)).
 *   alpha (object size), alpha_lb (stability lower bound of Lemma 4.2),
 *   vol_B (|B|, so that |B_alpha| = alpha^3 vol_B).
 *   r_dirs: all 0 for one basis shared by the three directions, or the sizes
 *   r_1 + r_2 + r_3 = r of one basis per direction (Sect. 4.1, the paper's
 *   PODP): the basis is W = [U_1 U_2 U_3], K, C, Me and G are the full
 *   W-space matrices (K_ij = U_i^H K U_j, Eq. (18)), column i of B is W^H C o_i,
 *   and the sweep solves direction i with the diagonal block only (Eq. (17)).
 * Pointers may be host or device memory; they are copied before return.
 * Returns MROM_EINVAL for r < 1, r > MROM_MAX_R, a null required pointer or
 * a non-finite scalar. */
#define MROM_MAX_R 112
typedef struct {
  int32_t r;
  const void* K;
  const void* K_in;
  const void* C;
  const void* Me;
  const void* B;
  const double* c00;
  const void* G;
  const double* N0;
  double alpha;
  double alpha_lb;
  double vol_B;
  int32_t r_dirs[3];
} mrom_reduced_desc;

mrom_status mrom_rom_from_reduced(mrom_handle h, const mrom_reduced_desc* desc, mrom_rom_t* out);
/* Batched form of mrom_rom_from_reduced (not in the paper; for loading a dictionary):
 * n_obj objects from descs (host array), handles written to out (host array of n_obj).
 * The objects share one stream-ordered device allocation, released with the last of
 * them (mrom_rom_free as usual); copies are asynchronous and the batch synchronises
 * once.  Same checks and errors as mrom_rom_from_reduced; the message names the first
 * failing object, and on any error no object is created.  1 <= n_obj <= 65535. */
mrom_status mrom_rom_from_reduced_batch(mrom_handle h, int32_t n_obj, const mrom_reduced_desc* descs,
                                        mrom_rom_t* out);

/* One object of a packed dictionary (host record).  Its region at byte offset `offset`
 * (a multiple of 16) of the packed buffer holds, complex128 row-major and back to back:
 * K (r x r), K_in (r x r, if has_kin), C (r x r), Me (r x r, if has_me), B (r x 3),
 * G ((2r+3)^2, if has_gram) -- the arrays of mrom_reduced_desc with one basis shared by the
 * directions.  N0 all zero for none. */
typedef struct {
  int32_t r;
  int32_t has_kin;
  int32_t has_me;
  int32_t has_gram;
  int64_t offset;
  double c00[9];
  double N0[9];
  double alpha;
  double alpha_lb;
  double vol_B;
} mrom_packed_obj;

/* As mrom_rom_from_reduced_batch for a dictionary held in one buffer (packed: host -- pinned
 * for speed -- or device, `bytes` long): one copy of the whole buffer into one device
 * allocation shared by the objects, the Gram splits of all objects in one launch and one
 * validity check, so the cost does not grow with one copy per array.  Regions must lie inside
 * the buffer.  Synchronous. */
mrom_status mrom_rom_from_packed(mrom_handle h, int32_t n_obj, const mrom_packed_obj* objs, const void* packed,
                                 size_t bytes, mrom_rom_t* out);
/* Basis size r of an object (per direction); 0 on a null object. */
int32_t mrom_rom_rank(mrom_rom_t rom);
/* Releases an object (stream-ordered on the stream the handle had when the object was created,
 * so that stream -- and the handle -- must still exist: release objects and plans before the
 * handle and before destroying that stream, also at process exit). */
void mrom_rom_free(mrom_rom_t rom);

/* mrom_rom_free of n objects (host array, entries set to NULL; NULL entries are skipped). */
void mrom_rom_free_batch(mrom_rom_t* roms, int32_t n);

/* ------------------------------------------------ off-line stage (project) */

/* The full-order problem of Sect. 3.1 as the projection needs it (all DEVICE
 * pointers, caller-owned, float64):
 *   K (Eq. (10a)): n x n CSR, int32 row pointers (n+1) and column indices, values;
 *   C (Eq. (10b)) and M (Eq. (10c)): lumped (diagonal) matrices, n values each
 *     (M may be NULL); eps scales M in A = K - i omega C + eps M;
 *   o: 3 x n, row i = coefficients of the total theta_i^(0) = theta~_i^(0) + e_i x xi
 *     (so the source is r_i = i omega C o_i, Eq. (9));
 *   X_diag: n positive values of a diagonal inner-product matrix X for the
 *     certificate's Riesz norm ||r||^2 = r^H X^-1 r (Lemma 4.2), or NULL.  With
 *     X = eps M + omega_min C, |a(v, v)| >= ||v||_X^2 / sqrt(2) for omega >= omega_min,
 *     so alpha_lb = 1/sqrt(2) is valid (a looser bound than the sparse X below);
 *   alpha, alpha_lb, vol_B, N0 (9 or NULL) as in mrom_reduced_desc;
 *   X_rowptr, X_col, X_val: a sparse real symmetric positive definite X (CSR, n x n,
 *     int32 indices), or NULL.  It takes precedence over X_diag.  With
 *     X = K + eps M + omega_min C, |a(v, v)| >= ||v||_X^2 / sqrt(2) for every
 *     omega >= omega_min (a(v, v) = v^H (K + eps M) v - i omega v^H C v), so alpha_lb =
 *     1/sqrt(2).  The library forms X^-1 Phi for the certificate's residual basis Phi
 *     by Jacobi-preconditioned conjugate gradients, every column together; a column
 *     stops at r^H D^-1 r <= X_tol^2 b^H D^-1 b (D = diag X; X_tol 0: 1e-13), and a
 *     column still iterating after X_max_iter iterations (0: 20000) or a breakdown
 *     (X not SPD) makes the call return MROM_ENOTCONVERGED.  Temporaries: 4 n (2r + 3)
 *     complex128.
 * No certificate when X_diag and X_rowptr are both NULL. */
typedef struct {
  int64_t n;
  const int32_t* K_rowptr;
  const int32_t* K_col;
  const double* K_val;
  const double* C_diag;
  const double* M_diag;
  double eps;
  const double* o;
  const double* X_diag;
  double alpha;
  double alpha_lb;
  double vol_B;
  const double* N0;
  const int32_t* X_rowptr;
  const int32_t* X_col;
  const double* X_val;
  double X_tol;
  int32_t X_max_iter;
} mrom_fom;

#define MROM_MAX_SNAPSHOTS 192

/* Off-line stage of Algorithm 1 with one basis for the three directions:
 * truncated SVD of the snapshot matrix [D_1 D_2 D_3] (Sect. 4.1, Eqs. (13)-(15))
 * and Galerkin projection (Sects. 4.2-4.3), producing a reduced object for
 * mrom_sweep.  D holds n_cols complex128 snapshot columns of length n, column c
 * at D + c * ldd (device, ldd >= n, n_cols <= MROM_MAX_SNAPSHOTS).  The SVD is
 * computed from the Hermitian Gram D^H D (Householder tridiagonalisation, then
 * divide and conquer on the tridiagonal up to MROM_MAX_R columns and implicit QL
 * above), so singular values below about 1e-8 s_1 are not resolved; the retained rank is
 * r = #{s_k / s_1 >= tol_sigma}, capped at r_max (if > 0) and MROM_MAX_R.
 * basis_in (device, n x r_in complex128 row-major, or NULL) skips the SVD and
 * projects onto the given basis.  sigma_out (host, n_cols values, or NULL)
 * receives the singular values; r_out (host, or NULL) the rank.  Synchronous:
 * allocates and frees its temporaries (about (3 r + 3) n complex values, plus
 * (2 r + 3) n when X_diag is given).  MROM_ENOTCONVERGED if the eigensolver
 * did not converge. */
mrom_status mrom_project(mrom_handle h, const mrom_fom* fom, const void* D, int64_t ldd, int32_t n_cols,
                         double tol_sigma, int32_t r_max, const void* basis_in, int32_t r_in, mrom_rom_t* out,
                         double* sigma_out, int32_t* r_out);

/* PODP in the relative permeability.  Sect. 4.2 notes that the precomputation of
 * Eqs. (17)-(19) carries over to parameters other than omega; here the parameter s
 * scales mu_r in every cell of the object (mu_r -> s mu_r).  K is linear in mu_r^-1
 * cell by cell (Eq. (10a)), so K(s) = (K - K_in) + K_in / s; theta~^(0) depends on s
 * through the static problem (K(s) + M_s) o~ = -K(s) x (Eq. (5)), and with it b, c00
 * and N0 (Eq. (6a)).  The conductivity needs no second parameter: it enters only
 * through nu = alpha^2 mu_0 omega sigma, so a conductivity scale is the sweep's
 * s_sigma.  All pointers are device pointers, owned by the caller. */
#define MROM_MAX_STATIC 64
typedef struct {
  const int32_t* Kin_rowptr; /* K_in: CSR n x n, the part of K carried by the object's cells (s = 1) */
  const int32_t* Kin_col;
  const double* Kin_val;
  const double* x;           /* 3 x n (row i at x + i n): the coefficients of e_i x xi */
  const double* kx;          /* 3 x n: K x at s = 1, K's columns of eliminated boundary edges included */
  const double* kx_in;       /* 3 x n: the part of kx carried by the object's cells */
  const double* M_static;    /* n: diagonal of the static problem's regularisation M_s */
  double vol_B_mu;           /* sum over the object's cells of |cell| / mu_r at s = 1 */
  const double* O;           /* static snapshots o~_i(s_l), real: n_o columns, column c at O + c * ldo */
  int64_t ldo;
  int32_t n_o;
  double tol_static;         /* truncation of the static snapshots' SVD, as tol_sigma */
} mrom_fom_mu;

/* As mrom_project (fom at s = 1; D holds snapshots q_i(omega_k, s_l) of the sampled
 * parameters, one basis U for all of them), plus K_in^r = U^H K_in U and the reduced
 * static problem: V from the SVD of O (rank m <= MROM_MAX_STATIC, r_out / m_out report
 * r and m), S(s) = V^H (K(s) + M_s) V, V^H K(s) x, U^H C V, V^H C V and V^H C x, so that
 * o~(s) ~= V y(s) with S(s) y = -V^H K(s) x.  The object's B, c00 and N0 are those of
 * the reduced static problem at s = 1; mrom_sweep and mrom_sweep_vjp evaluate it at
 * per-object s_mu with B, c00 and N0 following s_mu, and dL/ds_mu includes their
 * derivatives.  With fom->X_diag the object also keeps the Gram of
 * Phi_ext = [C x | C V | (K - K_in + eps M) U | K_in U | C U] in X^-1 (size 3 + m + 3 r), from
 * which the certificate of Lemma 4.2 follows at any s (the residual's source is the reduced
 * C (x + V y(s))); its stored certificate blocks are those of s = 1.  MROM_EINVAL if O has no
 * nonzero singular value.  Synchronous. */
mrom_status mrom_project_mu(mrom_handle h, const mrom_fom* fom, const mrom_fom_mu* mu, const void* D, int64_t ldd,
                            int32_t n_cols, double tol_sigma, int32_t r_max, mrom_rom_t* out, int32_t* r_out,
                            int32_t* m_out);

/* Rank m of an object's reduced static problem (0: none). */
int32_t mrom_rom_static_rank(mrom_rom_t rom);

/* The reduced static state of an object at the permeability scale s_mu (host outputs,
 * each optional): B (r x 3 complex128 row-major), c00, N0 (3 x 3), and their
 * derivatives with respect to s_mu.  Synchronous. */
mrom_status mrom_rom_mu_state(mrom_rom_t rom, double s_mu, void* B, double* c00, double* N0, void* dB, double* dc00,
                              double* dN0);

/* Full-order snapshots on the device: q_i(omega_k) solving Eq. (9),
 * (K + eps M - i omega_k C) q_i = i omega_k C o_i, for i = 1..3 and the n_w frequencies omega
 * (host), by the conjugate orthogonal conjugate gradient method (A is complex symmetric) with
 * Jacobi preconditioning, all 3 n_w right-hand sides iterated together (3 n_w <=
 * MROM_MAX_FOM_RHS).  Column 3 k + i of Q (device, complex128, column c at Q + c * ldq,
 * ldq >= n) receives q_i(omega_k), the snapshot layout of mrom_project.  A column stops when
 * ||D^-1/2 r|| <= tol ||D^-1/2 b|| (D = diag A); iters and res (host, 3 n_w each, or NULL)
 * receive the iteration counts and final scaled residuals.  MROM_ENOTCONVERGED if a column
 * did not reach tol within max_iter iterations or broke down (Q then holds the last iterates).
 * Temporaries: 5 n (3 n_w) complex128 and n (3 n_w) float64.  Synchronous. */
#define MROM_MAX_FOM_RHS 48
mrom_status mrom_fom_solve(mrom_handle h, const mrom_fom* fom, const double* omega, int32_t n_w, double tol,
                           int32_t max_iter, void* Q, int64_t ldq, int32_t* iters, double* res);

/* The static problem behind theta^(0) (Sect. 3, below Eq. (5): theta^(0) = e_i x xi + theta~^(0),
 * with theta~^(0) solving a regularised curl-curl problem when mu_r != 1), on the device:
 *   (K + M_s) o~_i = f_i,  i = 1..n_rhs,
 * K from fom (CSR), M_s (n, > 0) the regularisation's diagonal over all of Omega, and right-hand
 * sides with G^T f_i = 0 (e.g. f_i = -K x_i with K's columns of the eliminated boundary edges).
 * K vanishes on discrete gradients (K G = 0) while M_s is tiny, so the gradient part of o~ is fixed
 * only by G^T M_s o~ = 0, which a Krylov method on K + M_s resolves too slowly.  The call
 * therefore runs Jacobi PCG on K + M_s (which converges in the K part) and then removes the
 * gradient part exactly: o~ <- o~ - G y with (G^T M_s G) y = G^T M_s o~ (Jacobi PCG on the nodal
 * operator, applied as G^T (M_s (G y))).  The result solves the system and meets the gradient
 * condition, both to about tol; a sparse direct solve of K + M_s meets the latter only to
 * about cond(K + M_s) x rounding.
 *   G: n x n_nodes CSR (int32), the discrete gradient of the interior nodes (+-1 per edge);
 *   GT: its transpose (n_nodes x n CSR);  f, o: device, n_rhs x n (row i at + i n), float64;
 *   tol: relative preconditioned residual of both solves; iters (host, 2, or NULL): their
 *   iteration counts.  1 <= n_rhs <= MROM_MAX_STATIC_RHS.  Temporaries: 4 n + 2 n_nodes
 *   complex128 per right-hand side.  MROM_ENOTCONVERGED if a solve does not reach tol within
 *   max_iter iterations.  Synchronous. */
#define MROM_MAX_STATIC_RHS 8
mrom_status mrom_static_solve(mrom_handle h, const mrom_fom* fom, const double* M_s, int64_t n_nodes,
                              const int32_t* G_rowptr, const int32_t* G_col, const double* G_val,
                              const int32_t* GT_rowptr, const int32_t* GT_col, const double* GT_val,
                              const double* f, int32_t n_rhs, double tol, int32_t max_iter, double* o,
                              int32_t* iters);

/* Adaptive PODP, Algorithm 1 (Sect. 4.4), with one basis for the three directions.
 * Starting from ns0 >= 2 snapshots at omega0 (host, ns0 values) with their
 * 3 * ns0 full-order solution columns in D0 (length n each, column c at
 * D0 + c * n, host or device; any column order), repeat while
 * Lambda / |B_alpha| > tol_delta and k < max_k (k starts at 1):
 *   k <- k + 1; project (mrom_project with tol_sigma, r_max) and evaluate the
 *   certificate Delta on omega_out (device, n_out values, strictly increasing);
 *   Lambda_n = max over the output frequencies in [omega_n, omega_{n+1}) that are
 *   not snapshots of max_ij Delta_ij (ties: lowest frequency), Lambda = max_n;
 *   stop if Lambda / |B_alpha| <= tol_delta; else ask the callback for the
 *   full-order solutions at the frequencies of the n_star largest Lambda_n (one
 *   per interval), append them and re-project.  With 0 < theta <= 1 (the variant
 *   with a threshold described after Algorithm 1) the new frequencies are those of
 *   every interval with Lambda_n >= theta Lambda, the largest first and at most
 *   n_star per iteration; theta = 0 is the fixed n_star rule.
 * |B_alpha| = alpha^3 vol_B.  fom->X_diag is required (certificate).  The
 * callback receives n_new frequencies (host, ascending) and a HOST buffer of
 * 3 * n_new * n complex128 to fill: column j * 3 + i holds q_i(omega_new[j])
 * (Eq. (9)) at offset (j * 3 + i) * n; it returns 0 on success (anything else
 * stops the loop with MROM_ECALLBACK).  With cb NULL the library computes every
 * full-order snapshot itself with mrom_fom_solve (tolerance 1e-12), and D0 may be NULL
 * (then the initial snapshots are solved too).  Outputs: the final reduced object
 * (*out), Lambda after each certificate evaluation (lambda_hist, host, max_k
 * values, or NULL), the final k (k_done), the sorted snapshot frequencies
 * (omega_snap_out, host, ns0 + n_star (max_k - 1) values, or NULL) and their
 * number (ns_out).  Requires 3 (ns0 + n_star (max_k - 1)) <= MROM_MAX_SNAPSHOTS.
 * Synchronous; allocates its snapshot buffer. */
typedef int (*mrom_snapshot_cb)(void* user, int32_t n_new, const double* omega_new, void* D_new_host);
typedef struct {
  double tol_sigma;
  double tol_delta;
  int32_t n_star;
  int32_t max_k;
  int32_t r_max;
  double theta; /* 0, or a threshold in (0, 1] */
} mrom_adapt_opts;
mrom_status mrom_adapt(mrom_handle h, const mrom_fom* fom, const double* omega0, int32_t ns0, const void* D0,
                       mrom_snapshot_cb cb, void* user, const double* omega_out, int32_t n_out,
                       const mrom_adapt_opts* opts, mrom_rom_t* out, double* lambda_hist, int32_t* k_done,
                       double* omega_snap_out, int32_t* ns_out);

/* As mrom_project with one basis per direction, the paper's PODP (Sect. 4.1:
 * a TSVD of each D_i).  D holds 3 * n_s columns: n_s snapshots of direction 1,
 * then direction 2, then direction 3 (column c at D + c * ldd).  Each direction
 * is truncated with tol_sigma and r_max; r_1 + r_2 + r_3 <= MROM_MAX_R.  Or
 * basis_in (device, n x (r_1 + r_2 + r_3) complex128 row-major, columns
 * [U_1 U_2 U_3]) with r_dirs_in (host, 3).  sigma_out (host, 3 n_s, or NULL):
 * singular values per direction; r_dirs_out (host, 3, or NULL): the ranks.
 * The object's cross blocks give R_ij, I_ij of Eqs. (18)-(19) for i != j. */
mrom_status mrom_project_dirs(mrom_handle h, const mrom_fom* fom, const void* D, int64_t ldd, int32_t n_s,
                              double tol_sigma, int32_t r_max, const void* basis_in, const int32_t* r_dirs_in,
                              mrom_rom_t* out, double* sigma_out, int32_t* r_dirs_out);

/* Copy an object's reduced data to caller buffers (host or device; any may be
 * NULL): K, C, Me (r x r complex128; zeros when the object has no Me), B
 * (r x 3), c00 (9 float64, host), G ((2r+3)^2; MROM_EINVAL if the object has
 * no Gram matrix).  Synchronous. */
mrom_status mrom_rom_get(mrom_rom_t rom, void* K, void* C, void* Me, void* B, double* c00, void* G);

/* ------------------------------------------------------------------ sweep */

/* On-line stage of Algorithm 1 for a batch of objects (Sect. 4.3):
 * for every object o and frequency omega = omega[o*omega_stride + k]
 * (omega_stride = 0: one grid shared by all objects; n_w: one grid each),
 * solve (K + Me - i omega C) p_i = i omega b_i for i = 1..3 (Eq. (17)) and write
 *   R[o][k][i][j] = -alpha^3/4 Re(p_i^H K p_j) (+ N0_ij)              (Eq. (18))
 *   I[o][k][i][j] =  omega alpha^3/4 (c00_ij + Re(p_i^H C p_j
 *                    + b_i^H p_j + b_j^H p_i))                       (Eq. (19))
 *   Delta[o][k][i][j] (if Delta != NULL; Lemma 4.2, Eq. (20)):
 *     alpha^3/(8 alpha_lb) (||r_i||^2 + ||r_j||^2 + ||r_i - r_j||^2),
 *     ||r_i||^2 = w_i^H G w_i, w_i = [i omega e_i ; -p_i ; i omega p_i].
 * The reduced solves go through each object's Hermitian pencil or use LU
 * factorisation without pivoting (see mrom_set_solver); the latter is stable
 * here because A's Hermitian part after a pi/4 rotation, (K + omega C)/sqrt(2),
 * is positive definite for omega > 0.  omega must be finite and > 0; a
 * violation is reported by the next mrom_synchronize (outputs for that
 * frequency are NaN).  Delta != NULL requires every object to have a Gram
 * matrix (else MROM_EINVAL).  R, I, Delta are device pointers with room for
 * n_obj * n_w * 9 doubles; omega holds n_w (stride 0) or n_obj * n_w values.
 * s_sigma, s_mu (device, n_obj each, or NULL for 1): per-object conductivity
 * and permeability scales; s_sigma acts as omega -> s_sigma omega (nu is
 * linear in omega sigma).  With s_mu every object needs K_in: K(s) = K + (1/s - 1) K_in
 * (formed per call), and objects from mrom_project_mu take B, c00 and N0 of their reduced
 * static problem at s; Delta at s_mu needs objects from mrom_project_mu with a certificate
 * inner product (their extended Gram gives Lemma 4.2's Gram at s; MROM_ENOTSUP otherwise).
 * The per-call buffers of the scales take (r^2 + 5 r + 3 m + 2 r^2) complex128 per object. */
mrom_status mrom_sweep(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, const double* omega,
                       int32_t n_w, int32_t omega_stride, const double* s_sigma, const double* s_mu,
                       double* R, double* I, double* Delta);

/* Vector-Jacobian product of the sweep (not in the paper; gradients for
 * inverse problems and least-squares fits of material scales).  With the
 * forward model of mrom_sweep extended by a conductivity scale s_sigma
 * (omega -> s_sigma omega) and a permeability scale s_mu
 * (K(s_mu) = K + (1/s_mu - 1) K_in), and cotangents gR, gI ([n_obj][n_w][3][3],
 * device), it writes g_omega[o][k] = dL/domega (device, n_obj * n_w),
 * g_ssigma[o] = dL/ds_sigma and g_smu[o] = dL/ds_mu (device, n_obj each, or
 * NULL) for L = sum gR . R + gI . I, by an adjoint solve A^H Lambda = Z.  On the
 * pencil route (mrom_set_solver) the adjoint is diagonal in each object's
 * eigenbasis: Lambda = V (Lambda_K + i w)^-1 V^H Z, with V^H K_in V transformed
 * once per object when g_smu is wanted; objects that fail the pencil route's
 * accuracy gate, and every object on the LU route, use the same LU factors as
 * the forward solve (recomputed, not stored).  R and I (device, or NULL)
 * receive the forward values at these scales.  s_sigma, s_mu: device, n_obj
 * each, or NULL for 1; s_mu or g_smu require K_in on every object.
 * Asynchronous; allocates its tables stream-ordered. */
mrom_status mrom_sweep_vjp(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, const double* omega, int32_t n_w,
                           int32_t omega_stride, const double* s_sigma, const double* s_mu, const double* gR,
                           const double* gI, double* g_omega, double* g_ssigma, double* g_smu, double* R, double* I);

/* Mixed-precision sweep: the same outputs as mrom_sweep (no s_sigma, s_mu), with
 * the reduced systems eliminated in complex64 and refined n_refine times
 * (0..8) in float64: res = i omega B - (K + Me - i omega C) X in float64,
 * correction through the complex64 factors, X += d.  The quadratic forms of
 * Eqs. (18)-(19) and the certificate stay float64.  Each refinement step
 * multiplies the solution error by about kappa(A) * 6e-8; for the dictionary
 * spectra one step gives about 1e-7 relative and two give float64 accuracy.
 * Objects up to r = 96 (MROM_ENOTSUP above).  Asynchronous; allocates its task
 * tables stream-ordered. */
mrom_status mrom_sweep_mixed(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, const double* omega, int32_t n_w,
                             int32_t omega_stride, int32_t n_refine, double* R, double* I, double* Delta);

/* Certificate only: Delta as in mrom_sweep, without writing R and I. */
mrom_status mrom_certificate(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, const double* omega,
                             int32_t n_w, int32_t omega_stride, double* Delta);

/* A plan fixes a batch of objects and a frequency count once (device object
 * table, cost-sorted work list); mrom_plan_sweep then runs the same sweep as
 * mrom_sweep with no host-side preparation.  The plan keeps pointers to the
 * objects, which must outlive it.  mrom_plan_sweep allocates nothing and does
 * not wait on the host (stream-ordered memsets and kernel launches only), so a
 * caller may capture it on the handle's stream into a CUDA graph and replay the
 * graph (after one direct call, which sets the kernels' shared-memory limits);
 * a replay reads omega and writes R, I, Delta at the captured addresses, and
 * errors detected on the device surface at the next mrom_synchronize. */
mrom_status mrom_plan_create(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, int32_t n_w,
                             mrom_plan* out);
mrom_status mrom_plan_sweep(mrom_plan plan, const double* omega, int32_t omega_stride,
                            double* R, double* I, double* Delta);
/* Releases a plan (stream-ordered on its handle's stream; before the handle is destroyed). */
mrom_status mrom_plan_destroy(mrom_plan plan);
/* mrom_plan_sweep that also writes the rotation invariants of every evaluation (Sect. 1: the
 * eigenvalues of R~ = N0 + R and of I do not depend on the object's orientation), computed in the
 * sweep kernels' epilogue from the values they hold, so the 3 x 3 outputs need not be read back:
 * eig (device, [n_obj][n_w][6]): the eigenvalues of the symmetric part of R~ in ascending order,
 * then those of I (closed form, as mrom_invariants).  R, I and Delta may be NULL (then only the
 * invariants are written).  Same rules as mrom_plan_sweep otherwise. */
mrom_status mrom_plan_sweep_invariants(mrom_plan plan, const double* omega, int32_t omega_stride, double* R,
                                       double* I, double* Delta, double* eig);

/* Solver of the reduced systems for plans created (and one-shot sweeps run) after
 * this call.  MROM_SOLVER_AUTO (default): every object with one basis shared by
 * the directions goes through its Hermitian pencil (K + Me, C) -- per sweep, once
 * per object, C = L L^H, L^-1 (K + Me) L^-H = Z Lambda Z^H (Householder
 * tridiagonalisation and divide and conquer) and V = L^-H Z, after which each
 * frequency costs O(r) (the quadratic forms split at the poles into prefix and
 * suffix tables) instead of the O(r^3) elimination; same outputs up to rounding.
 * An object stays on the LU route when C is not numerically positive definite,
 * when ||C||_F ||L^-1||_F^2 > 1e6, when the error estimate
 * eps ||L^-1 (K + Me) L^-H||_F / omega_min exceeds 1e-11, when an eigenvalue of
 * the pencil is clearly negative, or when the eigensolver meets a non-finite
 * value (decided on the device, per sweep).  Objects with
 * one basis per direction always take the LU route.  MROM_SOLVER_LU: every
 * object takes the LU route. */
mrom_status mrom_set_solver(mrom_handle h, mrom_solver solver);

/* The sweep of a packed dictionary from HOST memory to HOST memory (Eqs. (17)-(19) and Lemma 4.2,
 * as mrom_plan_sweep): objects[n_obj] and packed/bytes as for mrom_rom_from_packed; omega (host,
 * n_w values shared by every object); R, I and Delta (host, [n_obj][n_w][3][3] float64; Delta may
 * be NULL: no certificate).  The objects are split into n_chunks contiguous groups of about equal
 * cost (1 <= n_chunks <= 16, at most n_obj); group c is uploaded, created, planned, swept and
 * read back on one of two library-owned streams while the other stream sweeps group c - 1, so the
 * host-device copies overlap the kernels of the neighbouring group.  Each group's preparation
 * kernels take about as long as their largest objects, so few groups pay best (two on a
 * 1000-object dictionary: 43.6 ms against 44.8 for one group and 60.3 for four).  Host buffers should be pinned
 * (pageable ones work and serialise the copies).  Synchronous: on return the outputs are on the
 * host, and every device allocation of the call is released.  The call orders itself after the
 * work already queued on the handle's stream.  Not reentrant on one handle.  Errors: as
 * mrom_rom_from_packed, mrom_plan_create and mrom_synchronize (the first failing group stops the
 * call; outputs of later groups are then unspecified); MROM_EINVAL for bad arguments. */
mrom_status mrom_sweep_host(mrom_handle h, int32_t n_obj, const mrom_packed_obj* objects, const void* packed,
                            size_t bytes, const double* omega, int32_t n_w, double* R, double* I, double* Delta,
                            int32_t n_chunks);

/* Objects that the last mrom_plan_sweep of this plan sent through the pencil
 * route (*n_pencil) and through LU elimination (*n_lu); either may be NULL.
 * Synchronous (waits for the handle's stream). */
mrom_status mrom_plan_solver_counts(mrom_plan plan, int32_t* n_pencil, int32_t* n_lu);

/* Stage timing of a plan's sweeps (not in the paper; for profiling).  enable != 0
 * creates CUDA events that every later mrom_plan_sweep records on the handle's
 * stream around its stages.  With stage_ms != NULL (host, 4 floats), waits for the
 * last sweep and writes the durations in ms of its pencil preparation, routing,
 * pencil sweep and LU sweep kernels (a plan without pencil objects has only the
 * last).  MROM_EINVAL when stage_ms is given and timing was never enabled. */
mrom_status mrom_plan_timing(mrom_plan plan, int32_t enable, float* stage_ms);

/* Autotuner: time every sweep launch configuration (threads per CTA x CTAs per
 * SM) on a sample of this batch (up to 96 objects x 200 frequencies) and make
 * the fastest the handle's configuration for later plans.  Blocks until done;
 * allocates and frees a scratch buffer.  *chosen (may be NULL) receives the
 * configuration index. */
mrom_status mrom_tune(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, int32_t n_w, int32_t* chosen);

/* The pencil route's launch mapping, picked by timing like mrom_tune: a plan sweep of a sample
 * of the objects (up to 2000 spread over the batch, up to 2048 log-spaced frequencies in
 * [1e1, 1e8]; the faster of two timed sweeps) with at most 8, 4, 2 or 1 frequency groups of 32
 * per sweep task (8 groups: one warp
 * per group runs every row of the object; fewer groups split the rows over the warps of a group
 * and reduce across them).  The fastest becomes the handle's cap for later plans (default 8);
 * *groups (may be NULL) receives it.  Results do not depend on the choice beyond rounding.
 * Blocks until done; allocates and frees a scratch buffer; device errors of the timed sweeps
 * are returned (mrom_synchronize). */
mrom_status mrom_tune_pencil(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, int32_t n_w, int32_t* groups);

/* ------------------------------------------------- rotation invariants */

/* Rotation-invariant features of a signature (Sect. 1: under a rotation Q of
 * the object each coefficient matrix becomes Q M Q^T, so its eigenvalues do
 * not depend on the orientation; dictionary matching compares the eigenvalues
 * of R~ = N0 + R and of I per frequency).  M: n real 3 x 3 matrices (device,
 * [n][3][3] row-major, e.g. the R or I output of mrom_sweep); eig: n x 3
 * eigenvalues of their symmetric parts in ascending order (device).  Closed form
 * per matrix (the trigonometric solution of the characteristic cubic for the
 * eigenvalue farthest from the others, deflation by its eigenvector, a 2 x 2
 * problem for the pair): absolute accuracy a few eps ||M||, repeated eigenvalues
 * included.  Asynchronous; MROM_EINVAL for n < 0 or null arrays with n > 0. */
mrom_status mrom_invariants(mrom_handle h, const double* M, int64_t n, double* eig);

/* ------------------------------------------------------------ measurement */

/* FP64 pipe throughput of the handle's device (not in the paper; the denominator of the FP64
 * kernels' roofline): independent fused multiply-add chains on every SM, timed with CUDA events
 * on the handle's stream.  *tflops receives 2 x the FMAs per second / 1e12, *ms (may be NULL)
 * the kernel's duration.  iters >= 1 (FMA steps per chain; 1 << 16 runs for about 10 ms).
 * Synchronous. */
mrom_status mrom_fp64_peak(mrom_handle h, int32_t iters, double* tflops, double* ms);

/* ------------------------------------------------------- allocation-free */

/* mrom_sweep without any device allocation.  Some callers cannot allocate
 * device memory while they run: a service that reserves its whole GPU memory
 * budget at start-up and forbids later allocations, an application whose own
 * allocator already owns the device memory, or a latency-critical loop in which
 * cudaMalloc / cudaFree would synchronise the device.  For them this entry point
 * computes exactly what mrom_sweep computes on the LU route (MROM_SOLVER_LU: same
 * kernel arithmetic, same outputs; the pencil route needs per-object tables that
 * scale with r^2 and is not offered here) and allocates nothing: the object
 * table, the task table, the work
 * counter and the workspace of systems too large for shared memory all live in
 * one fixed array of MROM_NOALLOC_SCRATCH_BYTES (64 MiB) of device memory inside
 * this library, which every GPU that loads the library holds until the process
 * exits.  The paper has no counterpart to this entry point.
 *  - Every call copies its object and task tables from host memory that lives
 *    only for the duration of the call.  To replay a sweep from a CUDA graph,
 *    use a plan (mrom_plan_create, mrom_plan_sweep).
 *  - The first call on a device looks up that array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *    With CUDA's lazy module loading (the default) the array is committed on a
 *    device when that first call loads this code, not when the library is
 *    loaded: a caller that reserves the rest of its memory budget afterwards
 *    makes one call at start-up first.  The address is kept per device index
 *    for the life of the process; after a cudaDeviceReset it is stale, so this
 *    entry point is not for processes that reset a device they used it on.
 *  - Every call reuses the same array (it keeps the previous call's contents):
 *    calls whose work overlaps on the GPU -- on different streams or handles of
 *    the same device -- race and corrupt each other's results; serialise them.
 *  - Arguments and output layout are those of mrom_sweep (without s_sigma and
 *    s_mu).  A batch whose tables and workspace do not fit the array is refused
 *    with MROM_EINVAL and a message giving the bytes needed; nothing is launched.
 *    The workspace shrinks the grid when needed, so only the tables (about 340
 *    bytes per object) bound the batch size. */
#define MROM_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
mrom_status mrom_sweep_noalloc(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, const double* omega,
                               int32_t n_w, int32_t omega_stride, double* R, double* I, double* Delta);

#ifdef __cplusplus
}
#endif

#endif /* MROM_H */

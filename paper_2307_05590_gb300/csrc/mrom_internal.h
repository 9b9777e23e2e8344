// Internal types shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mrom.h"

namespace mrom {

// Device status word bits (set by kernels with atomicOr, read by mrom_synchronize).
enum : int {
  kStatusBadOmega = 1,    // non-finite or non-positive frequency
  kStatusSingular = 2,    // zero or non-finite pivot
  kStatusTimeout = 4,     // a bounded wait gave up
  kStatusConfig = 8,      // a launch had less shared memory than a task needs (internal error)
};

// Per-object record read by the sweep kernels (device copy lives in a plan).
// All matrices are row-major complex128 (double2).
struct RomDev {
  const double2* K;     // r x r, used in R (Eq. (18)) and in A
  const double2* C;     // r x r
  const double2* Me;    // r x r or nullptr: U^H (eps M) U, added to A only
  const double2* Kin;   // r x r or nullptr: the permeability-dependent part of K (K(s_mu) = K + (1/s_mu - 1) K_in)
  const double2* B;     // r x 3: b_i in column i
  const double2* GKK;   // r x r  Gram block [(K+eps M)U]^H X^-1 [(K+eps M)U]
  const double2* GCC;   // r x r  Gram block (CU)^H X^-1 (CU)
  const double2* GSk;   // r x r  G_CK - G_KC (skew-Hermitian)
  const double2* gsK;   // 3 x r  rows of G: source column i against the K block
  const double2* gsC;   // 3 x r  rows of G: source column i against the C block
  double gss[9];        // Re G between source columns
  double c00[9];
  double N0[9];
  double alpha3;        // alpha^3
  double cert_scale;    // alpha^3 / (4 alpha_lb)
  int r;
  int has_cert;
  // Direction blocks of the basis W = [U_1 U_2 U_3] (Sect. 4.1: one TSVD per direction):
  // direction i's solution lives in rows [blk_lo[i], blk_hi[i]) and the reduced system uses
  // only the diagonal block A_ii.  A basis shared by the directions has [0, r) for all i.
  int per_dir;
  int blk_lo[3];
  int blk_hi[3];
  // PODP in mu_r (per call, when the permeability gradient is wanted): d/ds_mu of B, c00 and N0
  const double2* dB;  // r x 3 or nullptr
  double dc00[9];
  double dN0[9];
};

// Per-object data of the pencil route (pencil.cu), computed on the device by the
// preparation kernel of every sweep: eigenvalues lam (r, ascending), beta = V^H B (r x 3),
// gsh[k][q] = (gs_q V)[k] for the certificate rows of G (r x 6, or null), the transformed
// Gram blocks V^H G_X V for X = KK, CC, S interleaved per entry of the packed lower
// triangle with the diagonal halved (3 r (r+1)/2, or null) and V^H Me V (packed lower, or
// null), and for the sweep the pole-split tables of those Hermitian forms (pt, tb0, c0; null
// in adjoint tables; layout in pencil.cu).  F: frequency groups of 32 per sweep task.
struct PencilDev {
  double* lam;
  double2* beta;
  double* bbr;  // r x 6: Re(beta_ki^* beta_kj), (i, j) = 00 01 02 11 12 22
  double2* gsh;
  double2* Gh;
  double2* Eh;
  double2* Fh;  // V^H K_in V (packed lower, or null): the permeability gradient
  double2* dbeta;  // r x 3: V^H dB/ds_mu (or null)
  double2* pt;     // r (r+1)/2 entries x 21: per (m, k < m) the prefix/suffix polynomial tables
  double2* tb0;    // r x 12: per k the full suffix sums (KK, CC, iS, E) x 3
  double* c0;      // (r+1) x 24: per m the leading-block sums Re sum_{k,l<m} (KK, CC, iS, E) x 6
  int F;
  int pad;
};

// Per-object scratch of the pencil preparation: W = L^-H Q1 D (r x r), the tridiagonal's
// off-diagonal e (r), and the tridiagonal eigen-decomposition's workspace (3 r x r float64
// blocks; the first holds the eigenvectors Z2 afterwards).
struct PencilScratch {
  double2* W;
  double* e;
  double* work;
};

// One unit of work: S consecutive frequencies of one object.
struct SweepTask {
  int obj;
  int w0;
  int nw;
  int pad;
};

// Device tables of the pencil route for a batch of objects (pencil.cu): the eligible objects
// (one basis shared by the directions) in descending r, their data and preparation scratch,
// the routing tables and counters.  One stream-ordered allocation.
struct PencilTables {
  int n_pen = 0;                // eligible objects (0: no pencil route)
  int n_obj = 0, n_w = 0, rmax = 0;
  int prep_grid = 0, pen_grid = 0;
  size_t prep_ws_elems = 0, pen_smem = 0, pen_smem_vjp = 0;  // dynamic shared memory: sweep, adjoint
  void* block = nullptr;
  PencilDev* d_pens = nullptr;
  PencilScratch* d_scr = nullptr;
  int* d_order_pen = nullptr;   // eligible objects, descending r
  int* d_spen = nullptr;        // frequencies per pencil task, same order
  int* d_order_lu = nullptr;    // all objects in LU cost order
  int2* d_lu_info = nullptr;    // {S, matrices-in-global} of the LU kernel, per LU-order entry
  SweepTask* d_table_pen = nullptr;
  SweepTask* d_table_lu = nullptr;
  int* d_pen_ok = nullptr;
  int* d_counters = nullptr;    // tridiag, finish, pencil kernel, LU kernel, then the two route counts
  double2* d_prep_ws = nullptr;
};

}  // namespace mrom

// Opaque ABI objects.
struct mrom_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  int* d_status = nullptr;        // device status word
  int num_sms = 0;
  size_t smem_optin = 0;
  int64_t launches = 0;
  int sweep_cfg = -1;             // launch configuration for sweeps (-1: default)
  int projection_precision = 0;   // MROM_FP64 or MROM_MIXED for mrom_project's K U and Gram products
  int solver = 0;                 // MROM_SOLVER_AUTO or MROM_SOLVER_LU for plans and sweeps
  int pencil_fmax = 8;            // largest frequency-group count per pencil sweep task (1, 2, 4, 8)
  mrom_status pending = MROM_OK;  // host-detected asynchronous error
  std::string last_error;
  cudaStream_t aux[2] = {nullptr, nullptr};  // the pipelined host-buffer sweep's streams (lazily created)
};

namespace mrom {

// PODP in mu_r (a scale s of mu_r on the object): the reduced static problem of one object,
// S(s) y = -(kout + kin / s) with S(s) = Sout + Sin / s + Mv (m x m Hermitian, row-major), and
// the maps to B(s) = Bx + BV y, c00(s) = cxx + Re(cvx^H y + y^H cvx + y^H cvv y),
// N0(s) = (nB - mB / s) I + alpha^3/4 Re(y^H (Sout + Sin / s) y).  Per call the host sets the
// destinations of B(s) and dB/ds (r x 3) for the object.
struct MuDev {
  const double2 *Sout, *Sin, *Mv, *kout, *kin, *cvx, *cvv, *Bx, *BV;
  double cxx[9];
  double nB, mB, alpha3;
  int m, r;
  // certificate at s (or null): the Gram of Phi_ext = [C x | C V | (K_out + eps M) U | K_in U | C U]
  // in the certificate's inner product, next = 3 + m + 3 r rows and columns
  const double2* Gext;
  int next, pad;
  // per-call destinations (null where not wanted): B(s), dB/ds, y(s) (m x 3), and the
  // certificate's blocks at s (the split of Lemma 4.2's Gram used by the sweeps)
  double2* Bdst;
  double2* dBdst;
  double2* ydst;
  double2 *GKKdst, *GSkdst, *gsKdst, *gsCdst;
};

// Device buffer released at scope exit.
struct DevBuf {
  void* p = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// Per-object record of the LU-route adjoint kernel.
struct VjpDev {
  const double2 *K, *Kin, *C, *Me, *B;
  const double2* dB;  // d/ds_mu of B (PODP in mu_r) or nullptr
  double c00[9], N0[9], dc00[9], dN0[9];
  double alpha3;
  int r;
};

}  // namespace mrom

struct mrom_rom {
  mrom_ctx* ctx = nullptr;
  int r = 0;
  double alpha = 1.0, alpha_lb = 0.0, vol_B = 0.0;
  // device storage (one allocation, views below); objects of one batch share an allocation,
  // released (stream-ordered) with the last of them
  void* d_block = nullptr;
  struct SharedBlock {
    void* p = nullptr;
    int refs = 0;
    cudaStream_t stream = nullptr;
  }* shared = nullptr;
  double2 *K = nullptr, *Kin = nullptr, *C = nullptr, *Me = nullptr, *B = nullptr;
  double2 *GKK = nullptr, *GCC = nullptr, *GSk = nullptr, *gsK = nullptr, *gsC = nullptr;
  double2* G = nullptr;          // full Gram, kept for certificate-only consumers
  double gss[9] = {0};
  double c00[9] = {0};
  double N0[9] = {0};
  bool has_cert = false;
  bool has_kin = false;
  int r_dirs[3] = {0, 0, 0};  // per-direction basis sizes (all 0: one shared basis)
  // PODP in mu_r: the reduced static problem (device views in mu_block; mu.m == 0: none)
  mrom::MuDev mu{};
  void* mu_block = nullptr;
};

struct mrom_plan_s {
  mrom_ctx* ctx = nullptr;
  int cfg = 0;                      // sweep launch configuration
  int n_obj = 0, n_w = 0;
  bool all_cert = false;
  size_t smem_bytes = 0;
  int n_tasks = 0;
  int grid = 0;
  mrom::RomDev* d_objs = nullptr;
  mrom::SweepTask* d_tasks = nullptr;
  int* d_counter = nullptr;
  double2* d_workspace = nullptr;   // grid x ws_elems complex128, for tasks whose matrices are global
  size_t ws_elems = 0;
  mrom::PencilTables pen;           // pencil route (pen.n_pen > 0)
  // optional stage timing (mrom_plan_timing): events around prep, route, pencil sweep, LU sweep
  bool timing = false;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

namespace mrom {

// Set the handle's last error message and return the status.
mrom_status fail(mrom_ctx* h, mrom_status s, const std::string& msg);
mrom_status cuda_fail(mrom_ctx* h, cudaError_t e, const char* what);

// Sweep kernel launcher (sweep_fp64.cu).  A task's matrices live in shared memory
// (SweepTask.pad bit 0 clear) or in the CTA's slice of a global workspace (bit 0 set).
// Launch configurations differ in threads per CTA and CTAs per SM.
int sweep_fp64_num_configs();
int sweep_fp64_threads(int cfg);
int sweep_fp64_ctas_per_sm(int cfg);
// G (ma x mb complex128, row-major, ldg) = A^H diag(w) B for complex64 row-major A (n x ma) and
// B (n x mb), w (n, or null for 1), on the tensor cores (gram_tc.cu); ma, mb <= 112, A, B, w
// 16-byte aligned.  Synchronous.
cudaError_t tall_gram_tc(mrom_ctx* h, const float2* A, int ma, const float2* B, int mb, const float* w, int64_t n,
                         double2* G, int64_t ldg);

// Certificate inner product (riesz.cu): true when fom gives X_diag or a sparse X.
bool fom_has_certificate(const mrom_fom* fom);
// Y (n x nc, row-major complex128) = X^-1 Phi (same layout) for fom's sparse SPD X, by Jacobi PCG
// on all columns together; *iters_max (may be null) receives the largest iteration count.
// Synchronous.  MROM_ENOTCONVERGED when a column does not reach fom->X_tol.
mrom_status riesz_solve(mrom_ctx* h, const mrom_fom* fom, const double2* Phi, int nc, double2* Y, int* iters_max);

const void* sweep_fp64_symbol(int cfg);
// the compact-table instantiation that launch_sweep_fp64_implicit and launch_sweep_fp64_routed run
const void* sweep_fp64_implicit_symbol(int cfg);
size_t sweep_fp64_matrix_elems(int r);
size_t sweep_fp64_bytes_per_system(int r, bool matrix_in_smem);
cudaError_t sweep_fp64_configure(int cfg, size_t smem_bytes);
cudaError_t launch_sweep_fp64(int cfg, const RomDev* objs, const SweepTask* tasks, int n_tasks, int* counter,
                              const double* omega, int omega_stride, const double* s_sigma,
                              double* R, double* I, double* Delta, double* eig, int* status, int n_w, int grid,
                              size_t smem_bytes, double2* workspace, size_t ws_elems, cudaStream_t stream);

// Same sweep with the task list replaced by a compact per-object table (see
// implicit_task in sweep_fp64.cu); used by the allocation-free entry point.
cudaError_t launch_sweep_fp64_implicit(int cfg, const RomDev* objs, const SweepTask* table, int n_tasks,
                                       int* counter, const double* omega, int omega_stride, double* R,
                                       double* I, double* Delta, int* status, int n_w, int grid,
                                       size_t smem_bytes, double2* workspace, size_t ws_elems,
                                       cudaStream_t stream);
// Routed variant: the task table comes from the routing kernel and its header holds the
// task count (table[0].w0); s_sigma as in launch_sweep_fp64.
cudaError_t launch_sweep_fp64_routed(int cfg, const RomDev* objs, const SweepTask* table, int* counter,
                                     const double* omega, int omega_stride, const double* s_sigma, double* R,
                                     double* I, double* Delta, double* eig, int* status, int n_w, int grid,
                                     size_t smem_bytes, double2* workspace, size_t ws_elems, cudaStream_t stream);

// Pencil route (pencil.cu).
size_t pencil_sweep_smem_bytes();
// Tables for objs (host records; the device copy is passed to the kernels).  gram: tables of
// the forward sweep (certificate blocks of objects that have them, pole-split tables); kin:
// tables of the adjoint sweep with K_in transformed (permeability gradient).  order_lu / lu_info: every object in the LU kernel's cost order with its task
// shape {S, matrices-in-global}.  No eligible object: t->n_pen = 0 and nothing allocated.
mrom_status pencil_tables_create(mrom_ctx* h, const std::vector<RomDev>& objs, int n_w, bool gram, bool kin,
                                 const std::vector<int>& order_lu, const std::vector<int2>& lu_info, PencilTables* t);
void pencil_tables_destroy(PencilTables* t, cudaStream_t stream);
// Preparation (tridiagonalisation, divide and conquer, finishing) for one sweep; s_mu scales K_in as
// K + (1/s_mu - 1) K_in (NULL: no scale).  Resets the counters.  Then the routing kernel
// (pencil_tables_route) fills the pencil and LU task tables.
cudaError_t pencil_tables_prepare(mrom_ctx* h, const PencilTables& t, const RomDev* objs, const double* omega,
                                  int omega_stride, const double* s_sigma, const double* s_mu);
cudaError_t pencil_tables_route(mrom_ctx* h, const PencilTables& t);
size_t pencil_vjp_smem_bytes(int r, int F);
cudaError_t launch_pencil_vjp(const RomDev* objs, const PencilDev* pens, const SweepTask* table, int* counter,
                              const double* omega, int omega_stride, const double* s_sigma, const double* s_mu,
                              const double* gR, const double* gI, double* g_omega, double* g_mu_part, double* R,
                              double* I, int* status, int n_w, int grid, size_t smem_bytes, cudaStream_t stream);
cudaError_t launch_pencil_sweep(const RomDev* objs, const PencilDev* pens, const SweepTask* table, int* counter,
                                const double* omega, int omega_stride, const double* s_sigma, double* R,
                                double* I, double* Delta, double* eig, int* status, int n_w, int grid,
                                size_t smem_bytes, cudaStream_t stream);

// Builds the RomDev record of an object (api.cu).
RomDev rom_record(const mrom_rom* m);

// Full-order snapshots by COCG (fom_solve.cu): columns 3 k + i of Q (column c at Q + c ldq)
// receive q_i(omega[k]) for k < n_w (omega on the host).
mrom_status fom_solve(mrom_ctx* h, const mrom_fom* fom, const double* omega_host, int n_w, double tol, int max_iter,
                      double2* Q, int64_t ldq, int32_t* iters_out, double* res_out);

// PODP in mu_r (podp_mu.cu): for every object o with mus[o].m > 0, the static state at
// s_mu[o] (1 if s_mu is null): B(s) into mus[o].Bdst, dB/ds into mus[o].dBdst (when deriv), and
// c00, N0 (and dc00, dN0 when deriv) into recs[o] and vjp[o] (either array may be null).
// A non-positive pivot of the static system sets kStatusSingular in *status.
// m_max: the largest m in the batch (dynamic shared memory).
cudaError_t launch_mu_instance(const MuDev* mus, int n_obj, int m_max, const double* s_mu, bool deriv, RomDev* recs,
                               VjpDev* vjp, int* status, cudaStream_t stream);
// The certificate's Gram blocks of every object with mus[o].Gext at s_mu[o] (needs y(s) in
// mus[o].ydst from launch_mu_instance): G_KK(s), G_CK(s) - G_KC(s), g_sK(s), g_sC(s) into the
// destinations and gss(s) into recs[o].gss.
cudaError_t launch_mu_cert(const MuDev* mus, int n_obj, const double* s_mu, RomDev* recs, cudaStream_t stream);
// K(s) = K + (1/s - 1) K_in of each object with a K_in (jobs: {K, K_in, destination, r}).
struct ScaleKJob {
  const double2* K;
  const double2* Kin;
  double2* dst;
  int r, pad;
};
cudaError_t launch_scale_k(const ScaleKJob* jobs, int n_obj, int rmax, const double* s_mu, cudaStream_t stream);
size_t sweep_budget_bytes(const mrom_ctx* h, int cfg);
int sweep_config(const mrom_ctx* h);

// Certificate pre-processing of a Gram matrix (rom.cu).
cudaError_t launch_split_gram(const double2* G, int r, double2* GKK, double2* GCC, double2* GSk,
                              double2* gsK, double2* gsC, cudaStream_t stream);
// Sets *flag (device int) to 1 when any of the n doubles at x is not finite.
cudaError_t launch_nonfinite(const double* x, size_t n, int* flag, cudaStream_t stream);

}  // namespace mrom

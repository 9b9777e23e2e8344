// Riesz representers of the certificate's residual basis (Lemma 4.2): Y = X^-1 Phi for a sparse,
// real, symmetric positive definite inner-product matrix X, e.g. X = K + eps M + omega_min C, so
// that the certificate's Gram matrix is G = Phi^H Y and ||r^_i||^2 = w_i^H G w_i is the X^-1 norm
// of the full-order residual rho_i = Phi w_i.
//
// Preconditioned conjugate gradients with Jacobi preconditioning, every column of Phi iterated
// together.  X is real and symmetric positive definite, so for complex columns the Hermitian forms
// r^H D^-1 r and p^H X p are real and CG runs on C^n as on R^2n: alpha and beta are real.  Vectors
// are row-interleaved, V[row][column], so one pass over X's CSR serves every column; CTAs take
// groups of 32 columns (blockIdx.y), one warp spans a group's columns of one row, so every
// gathered neighbour row is one 512-byte contiguous read.  A column stops when its preconditioned
// residual satisfies r^H D^-1 r <= tol^2 b^H D^-1 b; on these matrices that quantity tracks the
// X-norm error of the iterate (both fall together until the rounding floor).  Per iteration:
// SpMV with the column partials of p^H q -> one-CTA reduction (alpha) -> update of y and r with
// the partials of r^H D^-1 r -> one-CTA reduction (beta, stop test) -> new direction.  All sums
// are in a fixed order (deterministic results).  Converged columns are skipped.
#include "mrom_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace mrom {
namespace {

constexpr int kRT = 256;          // threads per CTA
constexpr int kRW = 32;           // columns per group
constexpr int kRR = kRT / kRW;    // rows per CTA pass

struct RieszState {
  double rz;      // r^H D^-1 r of the current iterate
  double rz0;     // b^H D^-1 b
  double alpha;
  double beta;
  int active;     // 1 while the column iterates
  int iters;
  int breakdown;
  int pad;
};

// thread -> (row lr of the CTA pass, column c of the group; global column cg)
struct GroupMap {
  int c, lr, cg;
  bool on;
  __device__ explicit GroupMap(int nc) {
    c = threadIdx.x % kRW;
    lr = threadIdx.x / kRW;
    cg = blockIdx.y * kRW + c;
    on = cg < nc;
  }
};

// This CTA's column sums into part[group][block][c], rows summed in a fixed order.
__device__ void group_column_sum(double v, double* sh, double* __restrict__ part) {
  sh[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < kRW) {
    double s = 0.0;
    for (int l = 0; l < kRR; ++l) s += sh[l * kRW + threadIdx.x];
    part[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kRW + threadIdx.x] = s;
  }
}

// 1 / diag(X) (NaN for a non-positive diagonal, which then ends the column as a breakdown)
__global__ void riesz_dinv_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, int64_t n, double* __restrict__ dinv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] == i) d += val[k];
    dinv[i] = d > 0.0 ? 1.0 / d : __longlong_as_double(0x7ff8000000000000LL);
  }
}

// y = 0, r = b, p = D^-1 b; partials of b^H D^-1 b
__global__ void __launch_bounds__(kRT)
riesz_init_kernel(const double2* __restrict__ B, const double* __restrict__ dinv, int64_t n, int nc,
                  double2* __restrict__ Y, double2* __restrict__ Rv, double2* __restrict__ P,
                  double* __restrict__ part) {
  __shared__ double sh[kRT];
  const GroupMap m(nc);
  double acc = 0.0;
  if (m.on) {
    for (int64_t i = (int64_t)blockIdx.x * kRR + m.lr; i < n; i += (int64_t)gridDim.x * kRR) {
      const size_t e = (size_t)i * nc + m.cg;
      const double2 b = B[e];
      const double di = dinv[i];
      Y[e] = make_double2(0.0, 0.0);
      Rv[e] = b;
      P[e] = make_double2(di * b.x, di * b.y);
      acc += di * fma(b.x, b.x, b.y * b.y);
    }
  }
  group_column_sum(acc, sh, part);
}

// q = X p; partials of p^H q (real for symmetric X)
__global__ void __launch_bounds__(kRT)
riesz_spmv_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const double* __restrict__ val,
                  int64_t n, int nc, const RieszState* __restrict__ st, const double2* __restrict__ P,
                  double2* __restrict__ Q, double* __restrict__ part) {
  __shared__ double sh[kRT];
  const GroupMap m(nc);
  double acc = 0.0;
  if (m.on && st[m.cg].active) {
    for (int64_t i = (int64_t)blockIdx.x * kRR + m.lr; i < n; i += (int64_t)gridDim.x * kRR) {
      double2 q = make_double2(0.0, 0.0);
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const double v = val[k];
        const double2 pj = P[(size_t)col[k] * nc + m.cg];
        q.x = fma(v, pj.x, q.x);
        q.y = fma(v, pj.y, q.y);
      }
      const size_t e = (size_t)i * nc + m.cg;
      const double2 pi = P[e];
      Q[e] = q;
      acc += fma(pi.x, q.x, pi.y * q.y);
    }
  }
  group_column_sum(acc, sh, part);
}

// y += alpha p, r -= alpha q; partials of r^H D^-1 r
__global__ void __launch_bounds__(kRT)
riesz_update_kernel(int64_t n, int nc, const RieszState* __restrict__ st, const double* __restrict__ dinv,
                    double2* __restrict__ Y, double2* __restrict__ Rv, const double2* __restrict__ P,
                    const double2* __restrict__ Q, double* __restrict__ part) {
  __shared__ double sh[kRT];
  const GroupMap m(nc);
  double acc = 0.0;
  if (m.on && st[m.cg].active) {
    const double a = st[m.cg].alpha;
    for (int64_t i = (int64_t)blockIdx.x * kRR + m.lr; i < n; i += (int64_t)gridDim.x * kRR) {
      const size_t e = (size_t)i * nc + m.cg;
      const double2 p = P[e], q = Q[e];
      double2 y = Y[e], r = Rv[e];
      y.x = fma(a, p.x, y.x);
      y.y = fma(a, p.y, y.y);
      r.x = fma(-a, q.x, r.x);
      r.y = fma(-a, q.y, r.y);
      Y[e] = y;
      Rv[e] = r;
      acc += dinv[i] * fma(r.x, r.x, r.y * r.y);
    }
  }
  group_column_sum(acc, sh, part);
}

// p = D^-1 r + beta p
__global__ void __launch_bounds__(kRT)
riesz_direction_kernel(int64_t n, int nc, const RieszState* __restrict__ st, const double* __restrict__ dinv,
                       const double2* __restrict__ Rv, double2* __restrict__ P) {
  const GroupMap m(nc);
  if (!m.on || !st[m.cg].active) return;
  const double b = st[m.cg].beta;
  for (int64_t i = (int64_t)blockIdx.x * kRR + m.lr; i < n; i += (int64_t)gridDim.x * kRR) {
    const size_t e = (size_t)i * nc + m.cg;
    const double di = dinv[i];
    const double2 r = Rv[e], p = P[e];
    P[e] = make_double2(fma(b, p.x, di * r.x), fma(b, p.y, di * r.y));
  }
}

// mode 0 (after init): rz0; mode 1 (after SpMV): alpha; mode 2 (after update): beta and the stop
// test.  One warp per column sums part[group][b][c] over the blocks (lane-strided, then a shuffle
// tree: a fixed order); its lane 0 updates the column's state.
__global__ void __launch_bounds__(kRT)
riesz_reduce_kernel(const double* __restrict__ part, int nblk, int nc, int mode, double tol2,
                    RieszState* __restrict__ st) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = warp; c < nc; c += kRT / 32) {
    const double* pc = part + (size_t)(c / kRW) * nblk * kRW + (c % kRW);
    double v = 0.0;
    for (int b = lane; b < nblk; b += 32) v += pc[(size_t)b * kRW];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) {
      RieszState s = st[c];
      if (mode == 0) {
        s.rz = s.rz0 = v;
        s.active = v > 0.0 ? 1 : 0;
        s.breakdown = isfinite(v) ? 0 : 1;
        if (s.breakdown) s.active = 0;
        s.iters = 0;
        s.alpha = s.beta = 0.0;
      } else if (mode == 1) {
        if (s.active && !(v > 0.0 && isfinite(v))) {
          s.breakdown = 1;
          s.active = 0;
        }
        s.alpha = s.active ? s.rz / v : 0.0;
      } else {
        if (s.active) {
          s.beta = v / s.rz;
          s.rz = v;
          s.iters += 1;
          if (!isfinite(v)) {
            s.breakdown = 1;
            s.active = 0;
          } else if (!(v > tol2 * s.rz0)) {
            s.active = 0;  // converged
          }
        } else {
          s.beta = 0.0;
        }
      }
      st[c] = s;
    }
  }
}

// Columns of the SPD operator apply(P) -> Q: PCG on every column of B (row-interleaved, nc columns
// over n rows) with the Jacobi weights dinv; Y receives the solutions.  apply launches kernels that
// write Q = A P and the column partials of p^H q into part[group][block][c] with the grid
// (nblk, groups) of this driver, skipping columns whose state is inactive.
template <class Apply>
mrom_status pcg_columns(mrom_ctx* h, int64_t n, int nc, int nblk, const double* dinv, const double2* B, double2* Y,
                        double tol, int max_iter, Apply apply, int* iters_max, const char* what) {
  cudaStream_t st = h->stream;
  const int ngroups = (nc + kRW - 1) / kRW;
  const size_t nv = (size_t)n * nc;
  DevBuf vec, aux;
  cudaError_t e = cudaMalloc(&vec.p, 3 * nv * sizeof(double2));
  const size_t b_part = (size_t)ngroups * nblk * kRW * sizeof(double);
  if (e == cudaSuccess) e = cudaMalloc(&aux.p, b_part + nc * sizeof(RieszState) + 256);
  if (e != cudaSuccess) return cuda_fail(h, e, what);
  auto* Rv = static_cast<double2*>(vec.p);
  double2* P = Rv + nv;
  double2* Q = P + nv;
  auto* part = static_cast<double*>(aux.p);
  auto* sts = reinterpret_cast<RieszState*>(static_cast<char*>(aux.p) + b_part);
  const dim3 grid((unsigned)nblk, (unsigned)ngroups);
  riesz_init_kernel<<<grid, kRT, 0, st>>>(B, dinv, n, nc, Y, Rv, P, part);
  riesz_reduce_kernel<<<1, kRT, 0, st>>>(part, nblk, nc, 0, tol * tol, sts);
  h->launches += 2;
  e = cudaGetLastError();
  std::vector<RieszState> hs(nc);
  const int chunk = 25;
  auto iteration = [&]() {
    apply(sts, P, Q, part);
    riesz_reduce_kernel<<<1, kRT, 0, st>>>(part, nblk, nc, 1, tol * tol, sts);
    riesz_update_kernel<<<grid, kRT, 0, st>>>(n, nc, sts, dinv, Y, Rv, P, Q, part);
    riesz_reduce_kernel<<<1, kRT, 0, st>>>(part, nblk, nc, 2, tol * tol, sts);
    riesz_direction_kernel<<<grid, kRT, 0, st>>>(n, nc, sts, dinv, Rv, P);
  };
  // chunks of iterations captured once as a CUDA graph and replayed; direct launches on the
  // legacy default stream (which cannot be captured) or when the capture fails
  cudaGraphExec_t chunk_exec = nullptr;
  if (e == cudaSuccess && st != nullptr && max_iter >= chunk) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      for (int k = 0; k < chunk; ++k) iteration();
      const cudaError_t ce = cudaStreamEndCapture(st, &graph);
      if (ce == cudaSuccess && graph && cudaGraphInstantiate(&chunk_exec, graph, 0) != cudaSuccess)
        chunk_exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
  }
  int it = 0;
  bool done = false;
  while (e == cudaSuccess && !done && it < max_iter) {
    if (chunk_exec && it + chunk <= max_iter) {
      e = cudaGraphLaunch(chunk_exec, st);
      it += chunk;
      h->launches += (4 + Apply::kLaunches) * chunk;
    } else {
      const int k_end = std::min(max_iter, it + chunk);
      for (; it < k_end && e == cudaSuccess; ++it) {
        iteration();
        h->launches += 4 + Apply::kLaunches;
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), sts, nc * sizeof(RieszState), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    done = true;
    for (int c = 0; c < nc && e == cudaSuccess; ++c) done = done && !hs[c].active;
  }
  if (chunk_exec) cudaGraphExecDestroy(chunk_exec);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, what);
  int imax = 0;
  bool ok = true;
  for (int c = 0; c < nc; ++c) {
    imax = std::max(imax, hs[c].iters);
    ok = ok && !hs[c].active && !hs[c].breakdown;
  }
  if (iters_max) *iters_max = imax;
  if (!ok)
    return fail(h, MROM_ENOTCONVERGED,
                std::string(what) + ": PCG did not reach the tolerance within the iteration limit, or broke down "
                                    "(the matrix must be symmetric positive definite)");
  return MROM_OK;
}

// CTAs per column group: about 8 CTAs per SM over all groups, each over at least 64 rows
int pcg_blocks(const mrom_ctx* h, int64_t n, int nc) {
  const int ngroups = (nc + kRW - 1) / kRW;
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::max<int64_t>(1, (int64_t)h->num_sms * 8 / ngroups),
                                                     (n + 63) / 64));
}

// The CSR operator of pcg_columns
struct CsrApply {
  const int32_t *rowptr, *col;
  const double* val;
  int64_t n;
  int nc, nblk;
  cudaStream_t st;
  static constexpr int kLaunches = 1;
  void operator()(const RieszState* sts, const double2* P, double2* Q, double* part) const {
    const dim3 grid((unsigned)nblk, (unsigned)((nc + kRW - 1) / kRW));
    riesz_spmv_kernel<<<grid, kRT, 0, st>>>(rowptr, col, val, n, nc, sts, P, Q, part);
  }
};

// ---- static problem: (K + M_s) o = f with the gradient part fixed by M_s-orthogonality

// A = K + diag(M_s): K's values with M_s added on the diagonal entries
__global__ void static_matrix_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                     const double* __restrict__ kval, const double* __restrict__ ms, int64_t n,
                                     double* __restrict__ aval) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) aval[k] = kval[k] + (col[k] == i ? ms[i] : 0.0);
}

// V[i][c] = (f[c n + i], 0) for nc real columns
__global__ void real_rows_kernel(const double* __restrict__ f, int64_t n, int nc, double2* __restrict__ V) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nc;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / nc;
    const int c = (int)(idx - i * nc);
    V[idx] = make_double2(f[(int64_t)c * n + i], 0.0);
  }
}

// out[i][c] = w_i sum_k A[i][k] V[k][c] (CSR rows, w = null for 1), every column (no partials)
__global__ void __launch_bounds__(kRT)
csr_rows_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const double* __restrict__ val,
                const double* __restrict__ w, int64_t nrows, int nc, const double2* __restrict__ V,
                double2* __restrict__ out) {
  const GroupMap m(nc);
  if (!m.on) return;
  for (int64_t i = (int64_t)blockIdx.x * kRR + m.lr; i < nrows; i += (int64_t)gridDim.x * kRR) {
    double2 q = make_double2(0.0, 0.0);
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const double v = val[k];
      const double2 x = V[(size_t)col[k] * nc + m.cg];
      q.x = fma(v, x.x, q.x);
      q.y = fma(v, x.y, q.y);
    }
    const double s = w ? w[i] : 1.0;
    out[(size_t)i * nc + m.cg] = make_double2(s * q.x, s * q.y);
  }
}

// T = M_s (G P) on the edges, for the active columns of the nodal solve
__global__ void __launch_bounds__(kRT)
lap_edge_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const double* __restrict__ val,
                const double* __restrict__ ms, int64_t n_edges, int nc, const RieszState* __restrict__ st,
                const double2* __restrict__ P, double2* __restrict__ T) {
  const GroupMap m(nc);
  if (!m.on || !st[m.cg].active) return;
  for (int64_t i = (int64_t)blockIdx.x * kRR + m.lr; i < n_edges; i += (int64_t)gridDim.x * kRR) {
    double2 q = make_double2(0.0, 0.0);
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const double v = val[k];
      const double2 x = P[(size_t)col[k] * nc + m.cg];
      q.x = fma(v, x.x, q.x);
      q.y = fma(v, x.y, q.y);
    }
    T[(size_t)i * nc + m.cg] = make_double2(ms[i] * q.x, ms[i] * q.y);
  }
}

// Q = G^T T on the nodes (GT in CSR); partials of p^H q
__global__ void __launch_bounds__(kRT)
lap_node_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const double* __restrict__ val,
                int64_t n_nodes, int nc, const RieszState* __restrict__ st, const double2* __restrict__ T,
                const double2* __restrict__ P, double2* __restrict__ Q, double* __restrict__ part) {
  __shared__ double sh[kRT];
  const GroupMap m(nc);
  double acc = 0.0;
  if (m.on && st[m.cg].active) {
    for (int64_t j = (int64_t)blockIdx.x * kRR + m.lr; j < n_nodes; j += (int64_t)gridDim.x * kRR) {
      double2 q = make_double2(0.0, 0.0);
      for (int k = rowptr[j]; k < rowptr[j + 1]; ++k) {
        const double v = val[k];
        const double2 x = T[(size_t)col[k] * nc + m.cg];
        q.x = fma(v, x.x, q.x);
        q.y = fma(v, x.y, q.y);
      }
      const size_t e = (size_t)j * nc + m.cg;
      const double2 p = P[e];
      Q[e] = q;
      acc += fma(p.x, q.x, p.y * q.y);
    }
  }
  group_column_sum(acc, sh, part);
}

// 1 / diag(G^T M_s G): sum over the node's edges of GT^2 M_s
__global__ void lap_dinv_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ ms, int64_t n_nodes,
                                double* __restrict__ dinv) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n_nodes;
       j += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int k = rowptr[j]; k < rowptr[j + 1]; ++k) d += val[k] * val[k] * ms[col[k]];
    dinv[j] = d > 0.0 ? 1.0 / d : __longlong_as_double(0x7ff8000000000000LL);
  }
}

// T[i][c] = w_i V[i][c]
__global__ void scale_rows_kernel(const double* __restrict__ w, const double2* __restrict__ V, int64_t n, int nc,
                                  double2* __restrict__ T) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nc;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const double s = w[idx / nc];
    T[idx] = make_double2(s * V[idx].x, s * V[idx].y);
  }
}

// o[c n + i] = Re(Y[i][c] - GY[i][c])
__global__ void static_out_kernel(const double2* __restrict__ Y, const double2* __restrict__ GY, int64_t n, int nc,
                                  double* __restrict__ o) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nc;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / nc;
    const int c = (int)(idx - i * nc);
    o[(int64_t)c * n + i] = Y[idx].x - GY[idx].x;
  }
}

// The nodal operator G^T M_s G of pcg_columns (edge pass into T, then the node pass)
struct LapApply {
  const int32_t *g_rowptr, *g_col, *gt_rowptr, *gt_col;
  const double *g_val, *gt_val, *ms;
  int64_t n_edges, n_nodes;
  int nc, nblk, eblk;
  double2* T;
  cudaStream_t st;
  static constexpr int kLaunches = 2;
  void operator()(const RieszState* sts, const double2* P, double2* Q, double* part) const {
    const unsigned ng = (unsigned)((nc + kRW - 1) / kRW);
    lap_edge_kernel<<<dim3((unsigned)eblk, ng), kRT, 0, st>>>(g_rowptr, g_col, g_val, ms, n_edges, nc, sts, P, T);
    lap_node_kernel<<<dim3((unsigned)nblk, ng), kRT, 0, st>>>(gt_rowptr, gt_col, gt_val, n_nodes, nc, sts, T, P, Q,
                                                             part);
  }
};

}  // namespace

bool fom_has_certificate(const mrom_fom* fom) { return fom->X_diag != nullptr || fom->X_rowptr != nullptr; }

mrom_status riesz_solve(mrom_ctx* h, const mrom_fom* fom, const double2* Phi, int nc, double2* Y, int* iters_max) {
  const int64_t n = fom->n;
  const double tol = fom->X_tol > 0.0 ? fom->X_tol : 1e-13;
  const int max_iter = fom->X_max_iter > 0 ? fom->X_max_iter : 20000;
  const int nblk = pcg_blocks(h, n, nc);
  DevBuf dv;
  cudaError_t e = cudaMalloc(&dv.p, (size_t)n * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(h, e, "certificate inner product: allocation");
  auto* dinv = static_cast<double*>(dv.p);
  riesz_dinv_kernel<<<(unsigned)std::min<int64_t>(65535, (n + 255) / 256), 256, 0, h->stream>>>(
      fom->X_rowptr, fom->X_col, fom->X_val, n, dinv);
  ++h->launches;
  const CsrApply op{fom->X_rowptr, fom->X_col, fom->X_val, n, nc, nblk, h->stream};
  return pcg_columns(h, n, nc, nblk, dinv, Phi, Y, tol, max_iter, op, iters_max, "certificate inner product");
}

}  // namespace mrom

using namespace mrom;

extern "C" mrom_status mrom_static_solve(mrom_handle h, const mrom_fom* fom, const double* M_s, int64_t n_nodes,
                                         const int32_t* G_rowptr, const int32_t* G_col, const double* G_val,
                                         const int32_t* GT_rowptr, const int32_t* GT_col, const double* GT_val,
                                         const double* f, int32_t n_rhs, double tol, int32_t max_iter, double* o,
                                         int32_t* iters) {
  if (!h) return MROM_EINVAL;
  if (!fom || fom->n < 1 || !fom->K_rowptr || !fom->K_col || !fom->K_val)
    return fail(h, MROM_EINVAL, "mrom_static_solve: fom with n and K is required");
  if (!M_s || !G_rowptr || !G_col || !G_val || !GT_rowptr || !GT_col || !GT_val || !f || !o || n_nodes < 1)
    return fail(h, MROM_EINVAL, "mrom_static_solve: null argument or n_nodes < 1");
  if (n_rhs < 1 || n_rhs > MROM_MAX_STATIC_RHS || !(tol > 0.0) || !std::isfinite(tol) || max_iter < 1)
    return fail(h, MROM_EINVAL, "mrom_static_solve: 1 <= n_rhs <= MROM_MAX_STATIC_RHS, tol > 0, max_iter >= 1");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_static_solve: cudaSetDevice");
  const int64_t n = fom->n;
  const int nc = n_rhs;
  cudaStream_t st = h->stream;
  int32_t nnz = 0;
  e = cudaMemcpy(&nnz, fom->K_rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost);
  const size_t ne = (size_t)n * nc, nn = (size_t)n_nodes * nc;
  DevBuf aval, vecs, small;
  if (e == cudaSuccess) e = cudaMalloc(&aval.p, (size_t)std::max(nnz, 1) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&vecs.p, (4 * ne + 2 * nn) * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&small.p, ((size_t)n + (size_t)n_nodes) * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_static_solve: allocation");
  auto* F = static_cast<double2*>(vecs.p);
  double2* Y = F + ne;
  double2* T = Y + ne;
  double2* GY = T + ne;
  double2* Bn = GY + ne;
  double2* Yn = Bn + nn;
  auto* dinv = static_cast<double*>(small.p);
  double* dinv_n = dinv + n;
  auto* A = static_cast<double*>(aval.p);
  const auto g1 = [](int64_t work) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(65535, (work + 255) / 256)); };
  // 1. (K + M_s) o0 = f by PCG: converges in the K part; the gradient part of o0 is left undetermined
  static_matrix_kernel<<<g1(n), 256, 0, st>>>(fom->K_rowptr, fom->K_col, fom->K_val, M_s, n, A);
  riesz_dinv_kernel<<<g1(n), 256, 0, st>>>(fom->K_rowptr, fom->K_col, A, n, dinv);
  real_rows_kernel<<<g1(n * nc), 256, 0, st>>>(f, n, nc, F);
  h->launches += 3;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_static_solve: launch");
  const int nblk = pcg_blocks(h, n, nc);
  int it1 = 0, it2 = 0;
  mrom_status s = pcg_columns(h, n, nc, nblk, dinv, F, Y, tol, max_iter,
                              CsrApply{fom->K_rowptr, fom->K_col, A, n, nc, nblk, st}, &it1,
                              "mrom_static_solve (K + M_s)");
  if (s != MROM_OK) return s;
  // 2. remove the gradient part: (G^T M_s G) y = G^T M_s o0, o = o0 - G y
  const unsigned ng = (unsigned)((nc + kRW - 1) / kRW);
  scale_rows_kernel<<<g1(n * nc), 256, 0, st>>>(M_s, Y, n, nc, T);
  const int nblk_n = pcg_blocks(h, n_nodes, nc);
  csr_rows_kernel<<<dim3((unsigned)nblk_n, ng), kRT, 0, st>>>(GT_rowptr, GT_col, GT_val, nullptr, n_nodes, nc, T, Bn);
  lap_dinv_kernel<<<g1(n_nodes), 256, 0, st>>>(GT_rowptr, GT_col, GT_val, M_s, n_nodes, dinv_n);
  h->launches += 3;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_static_solve: launch");
  const LapApply lap{G_rowptr, G_col, GT_rowptr, GT_col, G_val, GT_val, M_s, n, n_nodes, nc, nblk_n, nblk, T, st};
  s = pcg_columns(h, n_nodes, nc, nblk_n, dinv_n, Bn, Yn, tol, max_iter, lap, &it2,
                  "mrom_static_solve (G^T M_s G)");
  if (s != MROM_OK) return s;
  csr_rows_kernel<<<dim3((unsigned)nblk, ng), kRT, 0, st>>>(G_rowptr, G_col, G_val, nullptr, n, nc, Yn, GY);
  static_out_kernel<<<g1(n * nc), 256, 0, st>>>(Y, GY, n, nc, o);
  h->launches += 2;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_static_solve");
  if (iters) {
    iters[0] = it1;
    iters[1] = it2;
  }
  return MROM_OK;
}

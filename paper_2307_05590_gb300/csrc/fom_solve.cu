// Full-order snapshot solves on the device: the systems of Eq. (9),
//   (K + eps M - i omega C) q_i(omega) = i omega C o_i,   i = 1..3,
// for every requested frequency at once, by the conjugate orthogonal conjugate gradient method
// (COCG: A is complex symmetric, A = A^T, so CG with the unconjugated bilinear form x^T y applies)
// with Jacobi preconditioning.  All 3 n_w right-hand sides iterate together in a row-interleaved
// layout X[row][column], so that one pass over K's CSR serves every column of an iteration.
//
// A column stops when its Jacobi-scaled residual ||D^-1/2 r|| falls below tol ||D^-1/2 b||
// (D = diag A).  The plain ||r|| / ||b|| is dominated by the conductor at high frequency, where
// the source i omega C o is large, and would stop before the exterior has converged.
// Per iteration: SpMV with the column partials of p^T q -> one-CTA reduction (alpha) -> update
// of x and r with the partials of r^T z and ||D^-1/2 r||^2 -> one-CTA reduction (beta, stop
// test) -> new direction.  Reductions are in a fixed order (deterministic results).
#include "mrom_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace mrom {
namespace {

constexpr int kFT = 256;        // threads per CTA
constexpr int kRedT = 256;      // threads of the one-CTA reductions

struct CocgState {
  double2 rho;      // r^T z of the current iterate
  double2 alpha;
  double2 beta;
  double nb;        // ||D^-1/2 b||^2
  double res;       // ||D^-1/2 r||^2
  int active;       // 1 while the column iterates
  int iters;
  int breakdown;
  int pad;
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double s = 1.0 / fma(b.x, b.x, b.y * b.y);
  return make_double2(fma(a.x, b.x, a.y * b.y) * s, fma(a.y, b.x, -a.x * b.y) * s);
}

// Thread layout of the row kernels: R = kFT / nc rows per CTA pass, thread t -> (row t / nc,
// column t % nc); threads t >= R nc idle.  The CTA strides over rows.
struct RowMap {
  int nc, R, c, lr;
  bool on;
  __device__ RowMap(int nc_) : nc(nc_) {
    R = kFT / nc;
    on = (int)threadIdx.x < R * nc;
    c = threadIdx.x % nc;
    lr = threadIdx.x / nc;
  }
};

// Column partial sums of this CTA into part[blockIdx.x][q][c] (nq quantities per column).
template <int NQ>
__device__ void block_column_sums(const RowMap& m, const double (&v)[NQ], double* sh, double* __restrict__ part) {
  for (int q = 0; q < NQ; ++q) sh[q * kFT + threadIdx.x] = m.on ? v[q] : 0.0;
  __syncthreads();
  for (int idx = threadIdx.x; idx < NQ * m.nc; idx += kFT) {
    const int q = idx / m.nc, c = idx - (idx / m.nc) * m.nc;
    double s = 0.0;
    for (int l = 0; l < m.R; ++l) s += sh[q * kFT + l * m.nc + c];
    part[((size_t)blockIdx.x * NQ + q) * m.nc + c] = s;
  }
  __syncthreads();
}

__global__ void kdiag_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const double* __restrict__ val, int64_t n, double* __restrict__ kd) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int k = rowptr[i]; k < rowptr[i + 1]; ++k)
      if (col[k] == i) v += val[k];
    kd[i] = v;
  }
}

__device__ __forceinline__ double2 diag_a(const double* kd, const double* cdiag, const double* mdiag, double eps,
                                          double w, int64_t i) {
  return make_double2(kd[i] + (mdiag ? eps * mdiag[i] : 0.0), -w * cdiag[i]);
}

// D^-1 and the residual weight 1/|d| per (row, column), once per solve (the iteration then
// needs no FP64 division or square root); x = 0, r = b = i w C o_dir, p = z = D^-1 r; partials
// of r^T z (complex) and ||D^-1/2 b||^2
__global__ void __launch_bounds__(kFT)
cocg_init_kernel(const double* __restrict__ omega, const double* __restrict__ kd, const double* __restrict__ cdiag,
                 const double* __restrict__ mdiag, double eps, const double* __restrict__ o, int64_t n, int nc,
                 double2* __restrict__ X, double2* __restrict__ Rv, double2* __restrict__ P,
                 double2* __restrict__ Dinv, double* __restrict__ Wt, double* __restrict__ part) {
  __shared__ double sh[3 * kFT];
  const RowMap m(nc);
  double acc[3] = {0.0, 0.0, 0.0};
  if (m.on) {
    const double w = omega[m.c / 3];
    const double* od = o + (int64_t)(m.c % 3) * n;
    for (int64_t i = (int64_t)blockIdx.x * m.R + m.lr; i < n; i += (int64_t)gridDim.x * m.R) {
      const double2 b = make_double2(0.0, w * cdiag[i] * od[i]);
      const double2 d = diag_a(kd, cdiag, mdiag, eps, w, i);
      const double id2 = 1.0 / fma(d.x, d.x, d.y * d.y);
      const double2 di = make_double2(d.x * id2, -d.y * id2);
      const double wt = sqrt(id2);  // 1 / |d|
      const double2 z = cmul(b, di);
      const size_t e = (size_t)i * nc + m.c;
      X[e] = make_double2(0.0, 0.0);
      Rv[e] = b;
      P[e] = z;
      Dinv[e] = di;
      Wt[e] = wt;
      const double2 rz = cmul(b, z);
      acc[0] += rz.x;
      acc[1] += rz.y;
      acc[2] += fma(b.x, b.x, b.y * b.y) * wt;
    }
  }
  block_column_sums<3>(m, acc, sh, part);
}

// q = A p (K by CSR, then the diagonal eps M - i w C); partials of p^T q
__global__ void __launch_bounds__(kFT)
cocg_spmv_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const double* __restrict__ val,
                 const double* __restrict__ omega, const double* __restrict__ cdiag, const double* __restrict__ mdiag,
                 double eps, int64_t n, int nc, const double2* __restrict__ P, double2* __restrict__ Q,
                 double* __restrict__ part) {
  __shared__ double sh[2 * kFT];
  const RowMap m(nc);
  double acc[2] = {0.0, 0.0};
  if (m.on) {
    const double w = omega[m.c / 3];
    for (int64_t i = (int64_t)blockIdx.x * m.R + m.lr; i < n; i += (int64_t)gridDim.x * m.R) {
      double2 q = make_double2(0.0, 0.0);
      for (int k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const double v = val[k];
        const double2 pj = P[(size_t)col[k] * nc + m.c];
        q.x = fma(v, pj.x, q.x);
        q.y = fma(v, pj.y, q.y);
      }
      const size_t e = (size_t)i * nc + m.c;
      const double2 pi = P[e];
      const double dr = mdiag ? eps * mdiag[i] : 0.0, di = -w * cdiag[i];
      q.x += dr * pi.x - di * pi.y;
      q.y += dr * pi.y + di * pi.x;
      Q[e] = q;
      const double2 pq = cmul(pi, q);
      acc[0] += pq.x;
      acc[1] += pq.y;
    }
  }
  block_column_sums<2>(m, acc, sh, part);
}

// x += alpha p, r -= alpha q; partials of r^T z (z = D^-1 r) and ||D^-1/2 r||^2
__global__ void __launch_bounds__(kFT)
cocg_update_kernel(int64_t n, int nc, const CocgState* __restrict__ st, const double2* __restrict__ Dinv,
                   const double* __restrict__ Wt, double2* __restrict__ X, double2* __restrict__ Rv,
                   const double2* __restrict__ P, const double2* __restrict__ Q, double* __restrict__ part) {
  __shared__ double sh[3 * kFT];
  const RowMap m(nc);
  double acc[3] = {0.0, 0.0, 0.0};
  if (m.on) {
    const double2 a = st[m.c].alpha;
    for (int64_t i = (int64_t)blockIdx.x * m.R + m.lr; i < n; i += (int64_t)gridDim.x * m.R) {
      const size_t e = (size_t)i * nc + m.c;
      const double2 p = P[e], q = Q[e];
      double2 x = X[e], r = Rv[e];
      const double2 ap = cmul(a, p), aq = cmul(a, q);
      x.x += ap.x;
      x.y += ap.y;
      r.x -= aq.x;
      r.y -= aq.y;
      X[e] = x;
      Rv[e] = r;
      const double2 rz = cmul(r, cmul(r, Dinv[e]));
      acc[0] += rz.x;
      acc[1] += rz.y;
      acc[2] += fma(r.x, r.x, r.y * r.y) * Wt[e];
    }
  }
  block_column_sums<3>(m, acc, sh, part);
}

// p = D^-1 r + beta p
__global__ void __launch_bounds__(kFT)
cocg_direction_kernel(int64_t n, int nc, const CocgState* __restrict__ st, const double2* __restrict__ Dinv,
                      const double2* __restrict__ Rv, double2* __restrict__ P) {
  const RowMap m(nc);
  if (!m.on) return;
  const double2 b = st[m.c].beta;
  for (int64_t i = (int64_t)blockIdx.x * m.R + m.lr; i < n; i += (int64_t)gridDim.x * m.R) {
    const size_t e = (size_t)i * nc + m.c;
    const double2 z = cmul(Rv[e], Dinv[e]);
    const double2 bp = cmul(b, P[e]);
    P[e] = make_double2(z.x + bp.x, z.y + bp.y);
  }
}

// mode 0 (after init): rho, nb;  mode 1 (after SpMV): alpha;  mode 2 (after update): beta, stop
// test.  One warp per (column, quantity) sums part[b][q][c] over the blocks (lane-strided, then a
// shuffle tree: a fixed order), then one thread per column updates its state.
__global__ void __launch_bounds__(kRedT)
cocg_reduce_kernel(const double* __restrict__ part, int nblk, int nc, int mode, double tol2,
                   CocgState* __restrict__ st) {
  __shared__ double vals[MROM_MAX_FOM_RHS * 3];
  const int nq = mode == 1 ? 2 : 3;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = warp; t < nc * nq; t += kRedT / 32) {
    const int c = t / nq, q = t - (t / nq) * nq;
    double v = 0.0;
    for (int b = lane; b < nblk; b += 32) v += part[((size_t)b * nq + q) * nc + c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) vals[t] = v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nc; c += kRedT) {
    const double* v = vals + c * nq;
    CocgState& s = st[c];
    if (mode == 0) {
      s.rho = make_double2(v[0], v[1]);
      s.nb = v[2];
      s.res = v[2];
      s.active = v[2] > 0.0 ? 1 : 0;
      s.iters = 0;
      s.breakdown = 0;
      s.alpha = s.beta = make_double2(0.0, 0.0);
    } else if (mode == 1) {
      const double2 pq = make_double2(v[0], v[1]);
      const double den = fma(pq.x, pq.x, pq.y * pq.y);
      if (s.active && !(den > 0.0 && isfinite(den))) {
        s.breakdown = 1;
        s.active = 0;
      }
      s.alpha = s.active ? cdiv(s.rho, pq) : make_double2(0.0, 0.0);
    } else {
      if (s.active) {
        const double2 rho = make_double2(v[0], v[1]);
        s.beta = cdiv(rho, s.rho);
        s.rho = rho;
        s.res = v[2];
        s.iters += 1;
        if (!(v[2] > tol2 * s.nb)) s.active = 0;  // converged (a NaN also stops it)
        if (!isfinite(v[2])) s.breakdown = 1;
      } else {
        s.beta = make_double2(0.0, 0.0);
      }
    }
  }
}

// Q[c * ldq + i] = X[i][c]
__global__ void cocg_store_kernel(const double2* __restrict__ X, int64_t n, int nc, double2* __restrict__ Qout,
                                  int64_t ldq) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n * nc;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / n, i = idx - (idx / n) * n;
    Qout[c * ldq + i] = X[(size_t)i * nc + c];
  }
}

}  // namespace

mrom_status fom_solve(mrom_ctx* h, const mrom_fom* fom, const double* omega_host, int n_w, double tol, int max_iter,
                      double2* Qout, int64_t ldq, int32_t* iters_out, double* res_out) {
  const int64_t n = fom->n;
  const int nc = 3 * n_w;
  cudaStream_t st = h->stream;
  const int R = kFT / nc;
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)h->num_sms * 8, (n + R - 1) / R));
  DevBuf vec, aux;
  const size_t nv = (size_t)n * nc;
  cudaError_t e = cudaMalloc(&vec.p, 5 * nv * sizeof(double2) + nv * sizeof(double));
  const size_t b_part = (size_t)nblk * 3 * nc * sizeof(double);
  const size_t b_aux = b_part + (size_t)n * sizeof(double) + nc * sizeof(CocgState) + n_w * sizeof(double) + 256;
  if (e == cudaSuccess) e = cudaMalloc(&aux.p, b_aux);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_fom_solve: allocation");
  auto* X = static_cast<double2*>(vec.p);
  double2* Rv = X + nv;
  double2* P = Rv + nv;
  double2* Q = P + nv;
  double2* Dinv = Q + nv;
  auto* Wt = reinterpret_cast<double*>(Dinv + nv);
  auto* part = static_cast<double*>(aux.p);
  auto* kd = reinterpret_cast<double*>(static_cast<char*>(aux.p) + b_part);
  auto* sts = reinterpret_cast<CocgState*>(kd + n);
  auto* om = reinterpret_cast<double*>(sts + nc);
  e = cudaMemcpyAsync(om, omega_host, n_w * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_fom_solve: upload");
  const unsigned g = (unsigned)std::min<int64_t>(65535, (n + 255) / 256);
  kdiag_kernel<<<g, 256, 0, st>>>(fom->K_rowptr, fom->K_col, fom->K_val, n, kd);
  cocg_init_kernel<<<nblk, kFT, 0, st>>>(om, kd, fom->C_diag, fom->M_diag, fom->eps, fom->o, n, nc, X, Rv, P, Dinv,
                                         Wt, part);
  cocg_reduce_kernel<<<1, kRedT, 0, st>>>(part, nblk, nc, 0, tol * tol, sts);
  h->launches += 3;
  e = cudaGetLastError();
  std::vector<CocgState> hs(nc);
  const int chunk = 25;
  auto iteration = [&]() {
    cocg_spmv_kernel<<<nblk, kFT, 0, st>>>(fom->K_rowptr, fom->K_col, fom->K_val, om, fom->C_diag, fom->M_diag,
                                           fom->eps, n, nc, P, Q, part);
    cocg_reduce_kernel<<<1, kRedT, 0, st>>>(part, nblk, nc, 1, tol * tol, sts);
    cocg_update_kernel<<<nblk, kFT, 0, st>>>(n, nc, sts, Dinv, Wt, X, Rv, P, Q, part);
    cocg_reduce_kernel<<<1, kRedT, 0, st>>>(part, nblk, nc, 2, tol * tol, sts);
    cocg_direction_kernel<<<nblk, kFT, 0, st>>>(n, nc, sts, Dinv, Rv, P);
  };
  // One chunk of iterations captured once as a CUDA graph and replayed (the launches of a
  // small problem cost more than its kernels); direct launches when the handle runs on the
  // legacy default stream (which cannot be captured) or the capture fails.
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
    cudaGetLastError();  // a failed capture leaves only the fallback
  }
  int it = 0;
  bool done = false;
  while (e == cudaSuccess && !done && it < max_iter) {
    if (chunk_exec && it + chunk <= max_iter) {
      e = cudaGraphLaunch(chunk_exec, st);
      it += chunk;
      h->launches += 5 * chunk;
    } else {
      const int k_end = std::min(max_iter, it + chunk);
      for (; it < k_end && e == cudaSuccess; ++it) {
        iteration();
        h->launches += 5;
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), sts, nc * sizeof(CocgState), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    done = true;
    for (int c = 0; c < nc && e == cudaSuccess; ++c) done = done && !hs[c].active;
  }
  if (chunk_exec) cudaGraphExecDestroy(chunk_exec);
  if (e == cudaSuccess) {
    cocg_store_kernel<<<(unsigned)std::min<int64_t>(65535 * 4, (n * nc + 255) / 256), 256, 0, st>>>(X, n, nc, Qout, ldq);
    ++h->launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_fom_solve");
  bool ok = true;
  for (int c = 0; c < nc; ++c) {
    if (iters_out) iters_out[c] = hs[c].iters;
    if (res_out) res_out[c] = hs[c].nb > 0.0 ? std::sqrt(hs[c].res / hs[c].nb) : 0.0;
    ok = ok && !hs[c].active && !hs[c].breakdown;
  }
  if (!ok) return fail(h, MROM_ENOTCONVERGED, "mrom_fom_solve: COCG did not reach the tolerance (or broke down)");
  return MROM_OK;
}

}  // namespace mrom

using namespace mrom;

extern "C" mrom_status mrom_fom_solve(mrom_handle h, const mrom_fom* fom, const double* omega, int32_t n_w,
                                      double tol, int32_t max_iter, void* Q, int64_t ldq, int32_t* iters,
                                      double* res) {
  if (!h) return MROM_EINVAL;
  if (!fom || !omega || !Q) return fail(h, MROM_EINVAL, "mrom_fom_solve: null argument");
  if (fom->n < 1 || !fom->K_rowptr || !fom->K_col || !fom->K_val || !fom->C_diag || !fom->o)
    return fail(h, MROM_EINVAL, "mrom_fom_solve: n, K, C_diag and o are required");
  if (n_w < 1 || 3 * n_w > MROM_MAX_FOM_RHS || ldq < fom->n)
    return fail(h, MROM_EINVAL, "mrom_fom_solve: 1 <= 3 n_w <= MROM_MAX_FOM_RHS and ldq >= n are required");
  if (!(tol > 0.0) || !std::isfinite(tol) || max_iter < 1)
    return fail(h, MROM_EINVAL, "mrom_fom_solve: tol > 0 and max_iter >= 1 are required");
  for (int k = 0; k < n_w; ++k)
    if (!(omega[k] > 0.0) || !std::isfinite(omega[k]))
      return fail(h, MROM_EINVAL, "mrom_fom_solve: frequencies must be finite and > 0");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_fom_solve: cudaSetDevice");
  return fom_solve(h, fom, omega, n_w, tol, max_iter, static_cast<double2*>(Q), ldq, iters, res);
}

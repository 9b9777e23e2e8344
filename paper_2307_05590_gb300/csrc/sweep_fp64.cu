// Batched reduced solves + Matrix-Method tensors + certificate, float64.
//
// One CTA processes a task: S consecutive frequencies of one reduced object
// (shared basis of size r, Remark 3.1 applied to all three directions).  For
// every frequency it
//   1. forms the augmented system [A | i omega B], A = K + Me - i omega C
//      (the reduced system of Eq. (17), with the three sources as columns);
//   2. eliminates without pivoting (A is sectorial: e^{i pi/4} A has the
//      positive definite Hermitian part (K + omega C)/sqrt(2), which bounds the
//      growth of Gaussian elimination);
//   3. back-substitutes the three right-hand sides;
//   4. forms y = M p for M in {K, C, G~(omega)} and the quadratic forms of
//      Eq. (18) (R), Eq. (19) (I) and, for the certificate of Lemma 4.2,
//      w_i^H G w_j = omega^2 Re G_ss + 2 Re(...) + p_i^H G~(omega) p_j with
//      G~(omega) = G_KK + omega^2 G_CC + i omega (G_CK - G_KC);
//   5. writes R, I and Delta.
// The FP64 pipe is the roofline of this kernel (GB300 executes two DFMA per
// clock per SM), so every phase spreads its work over all threads of the CTA,
// and all indexing runs on the integer pipes.  CTAs pull tasks from a
// cost-sorted list through an atomic counter (no waits).
#include "mrom_internal.h"

namespace mrom {
namespace {

constexpr int kThreads = 256;
constexpr int kRed = 36;  // reduced scalars per system

__device__ __forceinline__ double2 c_mac(double2 c, double2 a, double2 b) {   // c + a b
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 c_msub(double2 c, double2 a, double2 b) {  // c - a b
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// 1 / a with scaling against overflow; flags a zero or non-finite pivot.
__device__ __forceinline__ double2 c_recip(double2 a, int* status) {
  const double s = fmax(fabs(a.x), fabs(a.y));
  if (!(s > 0.0) || !isfinite(s)) {
    atomicOr(status, kStatusSingular);
    return make_double2(__longlong_as_double(0x7ff8000000000000LL), 0.0);
  }
  const double ax = a.x / s, ay = a.y / s;
  const double d = fma(ax, ax, ay * ay) * s;
  return make_double2(ax / d, -ay / d);
}

__device__ __forceinline__ void pair_ij(int q, int& i, int& j) {
  // (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)
  const int ti[6] = {0, 0, 0, 1, 1, 2};
  const int tj[6] = {0, 1, 2, 1, 2, 2};
  i = ti[q];
  j = tj[q];
}

__global__ void __launch_bounds__(kThreads, 1)
sweep_fp64_kernel(const RomDev* __restrict__ objs, const SweepTask* __restrict__ tasks, int n_tasks,
                  int* __restrict__ counter, const double* __restrict__ omega, int omega_stride,
                  const double* __restrict__ s_sigma, double* __restrict__ Rout,
                  double* __restrict__ Iout, double* __restrict__ Dout, int* __restrict__ status,
                  int n_w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task;
  const int tid = threadIdx.x;

  for (;;) {
    if (tid == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= n_tasks) break;

    const SweepTask task = tasks[t];
    const RomDev& ob = objs[task.obj];
    const int r = ob.r, S = task.nw, ld = r + 3;
    const bool want_cert = (Dout != nullptr) && ob.has_cert;

    const int am_elems = max(r * ld, 9 * r);
    double2* Am = reinterpret_cast<double2*>(smem_raw);          // S * am_elems
    double2* Pm = Am + (size_t)S * am_elems;                      // S * r * 3
    double2* Inv = Pm + (size_t)S * r * 3;                        // S * r
    double* Ws = reinterpret_cast<double*>(Inv + (size_t)S * r);  // S
    double* Red = Ws + S;                                         // S * kRed

    // ---- frequencies (s_sigma acts as omega -> s_sigma omega)
    const double ssig = s_sigma ? s_sigma[task.obj] : 1.0;
    for (int s = tid; s < S; s += kThreads) {
      const double w = omega[(size_t)task.obj * omega_stride + task.w0 + s] * ssig;
      const bool ok = (w > 0.0) && isfinite(w);
      if (!ok) atomicOr(status, kStatusBadOmega);
      Ws[s] = ok ? w : __longlong_as_double(0x7ff8000000000000LL);  // NaN outputs for a bad frequency
    }
    __syncthreads();

    // ---- 1. augmented systems [K + Me - i w C | i w B]
    for (int idx = tid; idx < S * r * ld; idx += kThreads) {
      const int s = idx / (r * ld);
      const int e = idx - s * r * ld;
      const int i = e / ld;
      const int j = e - i * ld;
      const double w = Ws[s];
      double2 v;
      if (j < r) {
        double2 k = ob.K[i * r + j];
        const double2 c = ob.C[i * r + j];
        if (ob.Me) {
          const double2 m = ob.Me[i * r + j];
          k.x += m.x;
          k.y += m.y;
        }
        v = make_double2(fma(w, c.y, k.x), fma(-w, c.x, k.y));
      } else {
        const double2 b = ob.B[i * 3 + (j - r)];
        v = make_double2(-w * b.y, w * b.x);
      }
      Am[(size_t)s * am_elems + e] = v;
      if (e == 0) Inv[(size_t)s * r] = c_recip(v, status);
    }
    __syncthreads();

    // ---- 2. elimination without pivoting (right-looking, RHS carried along)
    for (int k = 0; k < r - 1; ++k) {
      const int m = r - k - 1;
      for (int idx = tid; idx < S * m; idx += kThreads) {
        const int s = idx / m;
        const int i = k + 1 + (idx - s * m);
        double2* a = Am + (size_t)s * am_elems;
        a[i * ld + k] = c_mul(a[i * ld + k], Inv[(size_t)s * r + k]);
      }
      __syncthreads();
      const int nc = ld - k - 1;
      const int per = m * nc;
      for (int idx = tid; idx < S * per; idx += kThreads) {
        const int s = idx / per;
        const int e = idx - s * per;
        const int ii = e / nc;
        const int jj = e - ii * nc;
        const int i = k + 1 + ii, j = k + 1 + jj;
        double2* a = Am + (size_t)s * am_elems;
        const double2 v = c_msub(a[i * ld + j], a[i * ld + k], a[k * ld + j]);
        a[i * ld + j] = v;
        if (e == 0) Inv[(size_t)s * r + k + 1] = c_recip(v, status);
      }
      __syncthreads();
    }

    // ---- 3. back substitution, three right-hand sides
    for (int k = r - 1; k >= 0; --k) {
      for (int idx = tid; idx < S * 3; idx += kThreads) {
        const int s = idx / 3;
        const int j = idx - s * 3;
        const double2* a = Am + (size_t)s * am_elems;
        Pm[((size_t)s * r + k) * 3 + j] = c_mul(a[k * ld + r + j], Inv[(size_t)s * r + k]);
      }
      __syncthreads();
      if (k > 0) {
        const int per = k * 3;
        for (int idx = tid; idx < S * per; idx += kThreads) {
          const int s = idx / per;
          const int e = idx - s * per;
          const int i = e / 3;
          const int j = e - i * 3;
          double2* a = Am + (size_t)s * am_elems;
          a[i * ld + r + j] = c_msub(a[i * ld + r + j], a[i * ld + k], Pm[((size_t)s * r + k) * 3 + j]);
        }
        __syncthreads();
      }
    }

    // ---- 4a. y = M p for M in {K, C, G~(omega)}; Y overwrites the factors.
    // M is Hermitian, so M[a][b] = conj(M[b][a]) is read along a (coalesced).
    const int nm = want_cert ? 3 : 2;
    double2* Y = Am;  // Y[s][mm][a][j] at ((s*3 + mm)*r + a)*3 + j
    for (int idx = tid; idx < S * nm * r; idx += kThreads) {
      const int s = idx / (nm * r);
      const int e = idx - s * nm * r;
      const int mm = e / r;
      const int a = e - mm * r;
      const double2* p = Pm + (size_t)s * r * 3;
      double2 y0 = make_double2(0.0, 0.0), y1 = y0, y2 = y0;
      if (mm < 2) {
        const double2* M = (mm == 0) ? ob.K : ob.C;
        for (int b = 0; b < r; ++b) {
          double2 g = M[b * r + a];
          g.y = -g.y;
          y0 = c_mac(y0, g, p[b * 3 + 0]);
          y1 = c_mac(y1, g, p[b * 3 + 1]);
          y2 = c_mac(y2, g, p[b * 3 + 2]);
        }
      } else {
        const double w = Ws[s], w2 = w * w;
        for (int b = 0; b < r; ++b) {
          const double2 g = ob.GKK[b * r + a];
          const double2 c = ob.GCC[b * r + a];
          const double2 sk = ob.GSk[b * r + a];
          const double2 gt = make_double2(fma(w2, c.x, fma(-w, sk.y, g.x)),
                                          fma(-w2, c.y, fma(-w, sk.x, -g.y)));
          y0 = c_mac(y0, gt, p[b * 3 + 0]);
          y1 = c_mac(y1, gt, p[b * 3 + 1]);
          y2 = c_mac(y2, gt, p[b * 3 + 2]);
        }
      }
      double2* yo = Y + (((size_t)s * 3 + mm) * r + a) * 3;
      yo[0] = y0;
      yo[1] = y1;
      yo[2] = y2;
    }
    __syncthreads();

    // ---- 4b. reductions over the basis index a
    //  q 0..5  : Re(p_i^H K p_j)      q 6..11 : Re(p_i^H C p_j)
    //  q 12..17: Re(p_i^H G~ p_j)     q 18..26: Re(b_i^H p_j)
    //  q 27..35: Re((i w gsK_i + w^2 gsC_i) p_j)
    // without a certificate only the K and C forms (12) and Re(b_i^H p_j) (9) are needed
    const int nq = want_cert ? kRed : 21;
    for (int idx = tid; idx < S * nq; idx += kThreads) {
      const int s = idx / nq;
      int q = idx - s * nq;
      if (!want_cert && q >= 12) q += 6;  // skip the G~ block
      const double2* p = Pm + (size_t)s * r * 3;
      double acc = 0.0;
      if (q < 18) {
        int i, j;
        pair_ij(q % 6, i, j);
        const double2* y = Y + ((size_t)s * 3 + q / 6) * r * 3;
        for (int a = 0; a < r; ++a) {
          const double2 pa = p[a * 3 + i], ya = y[a * 3 + j];
          acc = fma(pa.x, ya.x, fma(pa.y, ya.y, acc));
        }
      } else if (q < 27) {
        const int i = (q - 18) / 3, j = (q - 18) % 3;
        for (int a = 0; a < r; ++a) {
          const double2 b = ob.B[a * 3 + i], pa = p[a * 3 + j];
          acc = fma(b.x, pa.x, fma(b.y, pa.y, acc));
        }
      } else {
        const int i = (q - 27) / 3, j = (q - 27) % 3;
        const double w = Ws[s], w2 = w * w;
        for (int a = 0; a < r; ++a) {
          const double2 gk = ob.gsK[i * r + a], gc = ob.gsC[i * r + a], pa = p[a * 3 + j];
          // coefficient (i w gk + w^2 gc); only the real part of its product with p is needed
          const double cx = fma(-w, gk.y, w2 * gc.x), cy = fma(w, gk.x, w2 * gc.y);
          acc = fma(cx, pa.x, fma(-cy, pa.y, acc));
        }
      }
      Red[(size_t)s * kRed + q] = acc;
    }
    __syncthreads();

    // ---- 5. outputs
    for (int idx = tid; idx < S * 9; idx += kThreads) {
      const int s = idx / 9;
      const int ij = idx - s * 9;
      const int i = ij / 3, j = ij - (ij / 3) * 3;
      const int lo = min(i, j), hi = max(i, j);
      const int q = (lo == 0) ? hi : (lo == 1 ? 2 + hi : 5);
      const double* red = Red + (size_t)s * kRed;
      const double w = Ws[s];
      const size_t o = ((size_t)task.obj * n_w + task.w0 + s) * 9 + ij;
      if (Rout) Rout[o] = fma(-0.25 * ob.alpha3, red[q], ob.N0[ij]);
      if (Iout) Iout[o] = 0.25 * ob.alpha3 * w * (ob.c00[ij] + red[6 + q] + red[18 + ij] + red[18 + j * 3 + i]);
      if (Dout) {
        if (want_cert) {
          const double w2 = w * w;
          const double cij = fma(w2, ob.gss[ij], red[12 + q] + red[27 + ij] + red[27 + j * 3 + i]);
          const int qi = (i == 0) ? 0 : (i == 1 ? 3 : 5), qj = (j == 0) ? 0 : (j == 1 ? 3 : 5);
          const double ni = fma(w2, ob.gss[i * 4], red[12 + qi] + 2.0 * red[27 + i * 4]);
          const double nj = fma(w2, ob.gss[j * 4], red[12 + qj] + 2.0 * red[27 + j * 4]);
          Dout[o] = ob.cert_scale * (ni + nj - cij);
        } else {
          Dout[o] = __longlong_as_double(0x7ff8000000000000LL);
        }
      }
    }
    // the next iteration's first barrier orders these reads before smem is reused
  }
}

}  // namespace

int sweep_fp64_threads() { return kThreads; }

const void* sweep_fp64_symbol() { return reinterpret_cast<const void*>(&sweep_fp64_kernel); }

size_t sweep_fp64_bytes_per_system(int r) {
  const size_t am = (size_t)(r * (r + 3) > 9 * r ? r * (r + 3) : 9 * r);
  return 16 * (am + 3 * (size_t)r + (size_t)r) + 8 * (1 + kRed);
}

cudaError_t sweep_fp64_configure(size_t smem_bytes) {
  return cudaFuncSetAttribute(sweep_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes);
}

cudaError_t launch_sweep_fp64(const RomDev* objs, const SweepTask* tasks, int n_tasks, int* counter,
                              const double* omega, int omega_stride, const double* s_sigma,
                              double* R, double* I, double* Delta, int* status, int n_w, int grid,
                              size_t smem_bytes, cudaStream_t stream) {
  sweep_fp64_kernel<<<grid, kThreads, smem_bytes, stream>>>(objs, tasks, n_tasks, counter, omega,
                                                            omega_stride, s_sigma, R, I, Delta,
                                                            status, n_w);
  return cudaGetLastError();
}

}  // namespace mrom

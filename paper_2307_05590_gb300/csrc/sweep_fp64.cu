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
//   3. back-substitutes the three right-hand sides (one warp per system and
//      right-hand side, warp-synchronous);
//   4. forms G~(omega) = G_KK + omega^2 G_CC + i omega (G_CK - G_KC) once (upper
//      triangle), then y = (L + D/2) p for each Hermitian M = L + D + L^H in
//      {K, C, G~}, so that Re(p_i^H M p_j) = Re(p_i^H y_j) + Re(p_j^H y_i) at
//      half the cost of M p, and reduces the quadratic forms of Eq. (18) (R),
//      Eq. (19) (I) and, for the certificate of Lemma 4.2,
//      w_i^H G w_j = omega^2 Re G_ss + 2 Re(...) + p_i^H G~ p_j;
//   5. writes R, I and Delta.
// The FP64 pipe is the roofline (GB300: two DFMA per clock per SM).  Several
// CTAs share an SM so that one CTA's barrier waits are filled by another's
// arithmetic; systems too large for their CTA's share of shared memory keep
// their matrices in an L2-resident global workspace.  Every phase splits its
// work into tasks of equal cost.  CTAs pull tasks from a cost-sorted list
// through an atomic counter (no waits).
#include "mrom_internal.h"
#include "eig3.cuh"

namespace mrom {
namespace {

constexpr int kRed = 45;    // reduced scalars per system
constexpr int kSplit = 4;   // partial sums per reduced scalar

__device__ __forceinline__ double2 c_msub(double2 c, double2 a, double2 b) {  // c - a b
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 c_conj_mac(double2 c, double2 a, double2 b) {  // c + conj(a) b
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
// 1 / a = conj(a) / |a|^2 (one division); flags a zero or non-finite pivot.
// |a|^2 stays in range for the pivot magnitudes of these systems (1e-150 .. 1e150).
__device__ __forceinline__ double2 c_recip(double2 a, int* status) {
  const double d = fma(a.x, a.x, a.y * a.y);
  if (!(d > 0.0) || !isfinite(d)) {
    atomicOr(status, kStatusSingular);
    return make_double2(__longlong_as_double(0x7ff8000000000000LL), 0.0);
  }
  const double id = 1.0 / d;
  return make_double2(a.x * id, -a.y * id);
}

// elements per system in the matrix buffer: the augmented system, later the
// y vectors (9 r) and the packed upper triangle of G~ (r (r+1) / 2)
__host__ __device__ __forceinline__ int matrix_elems(int r) {
  const int aug = r * (r + 3), forms = 9 * r + r * (r + 1) / 2;
  return aug > forms ? aug : forms;
}

// Compact task table: entry 0 is a header whose .obj holds the object count n; entries
// 1..n (objects in cost order) hold {object, frequencies per task S, first task index,
// matrices-in-global flag}.  Task t is chunk t - first of the entry whose range holds t.
__device__ __forceinline__ SweepTask implicit_task(const SweepTask* __restrict__ table, int n_w, int t) {
  const int n = table[0].obj;
  int lo = 1, hi = n + 1;  // table[lo].w0 <= t, and t < table[hi].w0 when hi <= n
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (table[mid].w0 <= t) lo = mid; else hi = mid;
  }
  const SweepTask e = table[lo];
  const int w0 = (t - e.w0) * e.nw;
  return SweepTask{e.obj, w0, min(e.nw, n_w - w0), e.pad & 1};
}

template <int THREADS, int MINB, bool IMPLICIT = false>
__global__ void __launch_bounds__(THREADS, MINB)
sweep_fp64_kernel(const RomDev* __restrict__ objs, const SweepTask* __restrict__ tasks, int n_tasks,
                  int* __restrict__ counter, const double* __restrict__ omega, int omega_stride,
                  const double* __restrict__ s_sigma, double* __restrict__ Rout,
                  double* __restrict__ Iout, double* __restrict__ Dout, double* __restrict__ Eout,
                  int* __restrict__ status, int n_w, double2* __restrict__ workspace, size_t ws_elems) {
  constexpr int kWarps = THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  if (IMPLICIT && n_tasks < 0) n_tasks = tasks[0].w0;  // routed table: count in the header

  for (;;) {
    if (tid == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= n_tasks) break;

    SweepTask task;
    if constexpr (IMPLICIT) {
      task = implicit_task(tasks, n_w, t);
    } else {
      task = tasks[t];
    }
    const RomDev& ob = objs[task.obj];
    const int r = ob.r, S = task.nw, ld = r + 3;
    const bool want_cert = (Dout != nullptr) && ob.has_cert;
    const bool in_global = (task.pad & 1) != 0;

    // buffers: matrices (shared memory, or this CTA's slice of the global workspace),
    // then solutions, pivot inverses, frequencies and partial reductions in shared memory
    const int am_elems = matrix_elems(r);
    double2* sp = reinterpret_cast<double2*>(smem_raw);
    double2* Am;
    if (in_global) {
      Am = workspace + (size_t)blockIdx.x * ws_elems;
    } else {
      Am = sp;
      sp += (size_t)S * am_elems;
    }
    double2* Pm = sp;
    double2* Inv = Pm + (size_t)S * r * 3;
    double* Ws = reinterpret_cast<double*>(Inv + (size_t)S * r);
    double* Red = Ws + S;  // S * kRed * kSplit

    // ---- frequencies (s_sigma acts as omega -> s_sigma omega)
    const double ssig = s_sigma ? s_sigma[task.obj] : 1.0;
    for (int s = tid; s < S; s += THREADS) {
      const double w = omega[(size_t)task.obj * omega_stride + task.w0 + s] * ssig;
      const bool ok = (w > 0.0) && isfinite(w);
      if (!ok) atomicOr(status, kStatusBadOmega);
      Ws[s] = ok ? w : __longlong_as_double(0x7ff8000000000000LL);  // NaN outputs for a bad frequency
    }
    __syncthreads();

    // ---- 1. augmented systems [K + Me - i w C | i w B]; with one basis per direction only the
    // diagonal blocks A_ii are kept and source i is restricted to block i (Eq. (17) per direction)
    const bool per_dir = ob.per_dir != 0;
    auto block_of = [&](int i) { return (int)(i >= ob.blk_lo[1]) + (int)(i >= ob.blk_lo[2]); };
    for (int idx = tid; idx < S * r * ld; idx += THREADS) {
      const int s = idx / (r * ld);
      const int e = idx - s * r * ld;
      const int i = e / ld;
      const int j = e - i * ld;
      const double w = Ws[s];
      double2 v = make_double2(0.0, 0.0);
      if (j < r) {
        if (!per_dir || block_of(i) == block_of(j)) {
          double2 k = ob.K[i * r + j];
          const double2 c = ob.C[i * r + j];
          if (ob.Me) {
            const double2 m = ob.Me[i * r + j];
            k.x += m.x;
            k.y += m.y;
          }
          v = make_double2(fma(w, c.y, k.x), fma(-w, c.x, k.y));
        }
      } else if (!per_dir || (i >= ob.blk_lo[j - r] && i < ob.blk_hi[j - r])) {
        const double2 b = ob.B[i * 3 + (j - r)];
        v = make_double2(-w * b.y, w * b.x);
      }
      Am[(size_t)s * am_elems + e] = v;
      // first pivot of the matrix and, per direction, of every block
      if (e == 0 || (per_dir && i == j && (i == ob.blk_lo[1] || i == ob.blk_lo[2])))
        Inv[(size_t)s * r + i] = c_recip(v, status);
    }
    __syncthreads();

    // ---- 2. elimination without pivoting (right-looking, right-hand sides carried along);
    // rows and columns of the pivot's direction block only (all of them for a shared basis)
    for (int k = 0; k < r - 1; ++k) {
      const int hi = per_dir ? (k < ob.blk_hi[0] ? ob.blk_hi[0] : (k < ob.blk_hi[1] ? ob.blk_hi[1] : ob.blk_hi[2])) : r;
      const int m = hi - k - 1;
      if (m == 0) continue;  // last pivot of a block (uniform across the CTA)
      for (int idx = tid; idx < S * m; idx += THREADS) {
        const int s = idx / m;
        const int i = k + 1 + (idx - s * m);
        double2* a = Am + (size_t)s * am_elems;
        a[i * ld + k] = c_mul(a[i * ld + k], Inv[(size_t)s * r + k]);
      }
      __syncthreads();
      const int nc = m + 3;  // the block's columns right of the pivot, then the three sources
      const int per = m * nc;
      const int total = S * per;
      // two independent elements per iteration: all loads are issued before either store
      for (int idx = tid; idx < total; idx += 2 * THREADS) {
        const int idx2 = idx + THREADS;
        const bool two = idx2 < total;
        const int s1 = idx / per;
        const int e1 = idx - s1 * per;
        const int c1 = e1 - (e1 / nc) * nc;
        const int i1 = k + 1 + e1 / nc, j1 = c1 < m ? k + 1 + c1 : r + (c1 - m);
        const int s2 = two ? idx2 / per : s1;
        const int e2 = two ? idx2 - s2 * per : e1;
        const int c2 = e2 - (e2 / nc) * nc;
        const int i2 = k + 1 + e2 / nc, j2 = c2 < m ? k + 1 + c2 : r + (c2 - m);
        double2* a1 = Am + (size_t)s1 * am_elems;
        double2* a2 = Am + (size_t)s2 * am_elems;
        const double2 x1 = a1[i1 * ld + j1], l1 = a1[i1 * ld + k], u1 = a1[k * ld + j1];
        const double2 x2 = a2[i2 * ld + j2], l2 = a2[i2 * ld + k], u2 = a2[k * ld + j2];
        const double2 v1 = c_msub(x1, l1, u1);
        const double2 v2 = c_msub(x2, l2, u2);
        a1[i1 * ld + j1] = v1;
        if (two) a2[i2 * ld + j2] = v2;
        if (e1 == 0) Inv[(size_t)s1 * r + k + 1] = c_recip(v1, status);
        if (two && e2 == 0) Inv[(size_t)s2 * r + k + 1] = c_recip(v2, status);
      }
      __syncthreads();
    }

    // ---- 3. back substitution: one warp per (system, right-hand side), warp-synchronous; the
    // solution of direction j is zero outside its block
    for (int sj = warp; sj < S * 3; sj += kWarps) {
      const int s = sj / 3, j = sj - (sj / 3) * 3;
      double2* a = Am + (size_t)s * am_elems;
      const double2* inv = Inv + (size_t)s * r;
      double2* p = Pm + (size_t)s * r * 3;
      const int lo = ob.blk_lo[j], hi = ob.blk_hi[j];
      for (int k = lane; k < r; k += 32)
        if (k < lo || k >= hi) p[k * 3 + j] = make_double2(0.0, 0.0);
      for (int k = hi - 1; k >= lo; --k) {
        const double2 x = c_mul(a[k * ld + r + j], inv[k]);  // every lane reads the same y_k
        for (int i = lo + lane; i < k; i += 32) a[i * ld + r + j] = c_msub(a[i * ld + r + j], a[i * ld + k], x);
        if (lane == 0) p[k * 3 + j] = x;
        __syncwarp();
      }
    }
    __syncthreads();

    // The matrix buffer of system s now holds Y[mm][a][j] (9 r entries) followed by the
    // packed upper triangle of G~ (row b holds columns a = b..r-1).
    const int nm = want_cert ? 3 : 2;
    const int half = (r + 1) / 2;
    auto tri = [r](int b, int a) { return b * r - (b * (b - 1)) / 2 + (a - b); };

    // ---- 4a. G~(omega) upper triangle, once per system
    if (want_cert) {
      const int ntri = r * (r + 1) / 2;
      for (int idx = tid; idx < S * ntri; idx += THREADS) {
        const int s = idx / ntri;
        int e = idx - s * ntri;
        // row b of the packed triangle holds r - b entries
        int b = 0;
        while (e >= r - b) {
          e -= r - b;
          ++b;
        }
        const int a = b + e;
        const double w = Ws[s], w2 = w * w;
        const double2 gk = ob.GKK[b * r + a], gc = ob.GCC[b * r + a], sk = ob.GSk[b * r + a];
        // G~_ba = G_KK,ba + w^2 G_CC,ba + i w GSk_ba
        Am[(size_t)s * am_elems + 9 * r + e + tri(b, b)] =
            make_double2(fma(w2, gc.x, fma(-w, sk.y, gk.x)), fma(w2, gc.y, fma(w, sk.x, gk.y)));
      }
      __syncthreads();
    }

    // ---- 4b. y_j = (L + D/2) p_j, one task per (system, matrix, row pair, j); rows a and
    // r-1-a share a task so that every task costs r + 1 complex multiply-adds.  The lower
    // triangle is read through M[a][b] = conj(M[b][a]) along a (coalesced).
    for (int idx = tid; idx < S * nm * half * 3; idx += THREADS) {
      const int s = idx / (nm * half * 3);
      int e = idx - s * nm * half * 3;
      const int mm = e / (half * 3);
      e -= mm * half * 3;
      const int pr = e / 3;
      const int j = e - pr * 3;
      const double2* p = Pm + (size_t)s * r * 3;
      double2* ys = Am + (size_t)s * am_elems;
      const double2* gt = ys + 9 * r;
      const double2* M = mm == 0 ? ob.K : ob.C;
      for (int side = 0; side < 2; ++side) {
        const int a = side == 0 ? pr : r - 1 - pr;
        if (side == 1 && a == pr) break;
        double2 y = make_double2(0.0, 0.0);
        if (mm < 2) {
          for (int b = 0; b < a; ++b) y = c_conj_mac(y, M[b * r + a], p[b * 3 + j]);
          const double2 d = M[a * r + a];
          y = c_conj_mac(y, make_double2(0.5 * d.x, 0.5 * d.y), p[a * 3 + j]);
        } else {
          for (int b = 0; b < a; ++b) y = c_conj_mac(y, gt[tri(b, a)], p[b * 3 + j]);
          const double2 d = gt[tri(a, a)];
          y = c_conj_mac(y, make_double2(0.5 * d.x, 0.5 * d.y), p[a * 3 + j]);
        }
        ys[(mm * r + a) * 3 + j] = y;
      }
    }
    __syncthreads();

    // ---- 4c. partial reductions over the basis index a (all nine (i, j); symmetrised in 5)
    //  q  0.. 8: Re(p_i^H y^K_j)   q  9..17: Re(p_i^H y^C_j)   q 18..26: Re(p_i^H y^G_j)
    //  q 27..35: Re(b_i^H p_j)     q 36..44: Re((i w gsK_i + w^2 gsC_i) p_j)
    // without a certificate only q 0..17 and 27..35 are formed
    const int nq = want_cert ? kRed : 27;
    for (int idx = tid; idx < S * nq * kSplit; idx += THREADS) {
      const int s = idx / (nq * kSplit);
      const int e = idx - s * nq * kSplit;
      int q = e / kSplit;
      const int part = e - q * kSplit;
      if (!want_cert && q >= 18) q += 9;
      const int a0 = (r * part) / kSplit, a1 = (r * (part + 1)) / kSplit;
      const double2* p = Pm + (size_t)s * r * 3;
      double acc = 0.0;
      if (q < 27) {
        const int i = (q % 9) / 3, j = q % 3;
        const double2* y = Am + (size_t)s * am_elems + (q / 9) * r * 3;
        for (int a = a0; a < a1; ++a) {
          const double2 pa = p[a * 3 + i], ya = y[a * 3 + j];
          acc = fma(pa.x, ya.x, fma(pa.y, ya.y, acc));
        }
      } else if (q < 36) {
        const int i = (q - 27) / 3, j = (q - 27) % 3;
        for (int a = a0; a < a1; ++a) {
          const double2 b = ob.B[a * 3 + i], pa = p[a * 3 + j];
          acc = fma(b.x, pa.x, fma(b.y, pa.y, acc));
        }
      } else {
        const int i = (q - 36) / 3, j = (q - 36) % 3;
        const double w = Ws[s], w2 = w * w;
        for (int a = a0; a < a1; ++a) {
          const double2 gk = ob.gsK[i * r + a], gc = ob.gsC[i * r + a], pa = p[a * 3 + j];
          // coefficient (i w gk + w^2 gc); only the real part of its product with p is needed
          const double cx = fma(-w, gk.y, w2 * gc.x), cy = fma(w, gk.x, w2 * gc.y);
          acc = fma(cx, pa.x, fma(-cy, pa.y, acc));
        }
      }
      Red[((size_t)s * kRed + q) * kSplit + part] = acc;
    }
    __syncthreads();

    // ---- 5. outputs
    for (int idx = tid; idx < S * 9; idx += THREADS) {
      const int s = idx / 9;
      const int ij = idx - s * 9;
      const int i = ij / 3, j = ij - (ij / 3) * 3;
      const int ji = j * 3 + i;
      const double* rp = Red + (size_t)s * kRed * kSplit;
      auto red = [rp](int q) {
        double v = 0.0;
#pragma unroll
        for (int k = 0; k < kSplit; ++k) v += rp[q * kSplit + k];
        return v;
      };
      const double w = Ws[s];
      const size_t o = ((size_t)task.obj * n_w + task.w0 + s) * 9 + ij;
      if (Rout) Rout[o] = fma(-0.25 * ob.alpha3, red(ij) + red(ji), ob.N0[ij]);
      if (Iout)
        Iout[o] = 0.25 * ob.alpha3 * w * (ob.c00[ij] + red(9 + ij) + red(9 + ji) + red(27 + ij) + red(27 + ji));
      if (Dout) {
        if (want_cert) {
          const double w2 = w * w;
          const double cij = fma(w2, ob.gss[ij], red(18 + ij) + red(18 + ji) + red(36 + ij) + red(36 + ji));
          const double ni = fma(w2, ob.gss[i * 4], 2.0 * (red(18 + i * 4) + red(36 + i * 4)));
          const double nj = fma(w2, ob.gss[j * 4], 2.0 * (red(18 + j * 4) + red(36 + j * 4)));
          Dout[o] = ob.cert_scale * (ni + nj - cij);
        } else {
          Dout[o] = __longlong_as_double(0x7ff8000000000000LL);
        }
      }
    }
    // ---- rotation invariants: eigenvalues of the symmetric parts of R~ and I (one thread per
    // frequency and matrix)
    if (Eout) {
      for (int idx = tid; idx < 2 * S; idx += THREADS) {
        const int s = idx >> 1, is_i = idx & 1;
        const double* rp = Red + (size_t)s * kRed * kSplit;
        auto red = [rp](int q) {
          double v = 0.0;
#pragma unroll
          for (int k = 0; k < kSplit; ++k) v += rp[q * kSplit + k];
          return v;
        };
        const double w = Ws[s];
        double Mp[6];  // packed (00, 01, 02, 11, 12, 22)
#pragma unroll
        for (int sym = 0; sym < 6; ++sym) {
          const int i = sym < 3 ? 0 : (sym < 5 ? 1 : 2), j = sym < 3 ? sym : (sym < 5 ? sym - 2 : 2);
          const int ij = i * 3 + j, ji = j * 3 + i;
          Mp[sym] = is_i ? 0.25 * ob.alpha3 * w *
                               (0.5 * (ob.c00[ij] + ob.c00[ji]) + red(9 + ij) + red(9 + ji) + red(27 + ij) + red(27 + ji))
                         : fma(-0.25 * ob.alpha3, red(ij) + red(ji), 0.5 * (ob.N0[ij] + ob.N0[ji]));
        }
        double* e = Eout + ((size_t)task.obj * n_w + task.w0 + s) * 6 + 3 * is_i;
        sym3_eig(Mp[0], Mp[3], Mp[5], Mp[1], Mp[2], Mp[4], e[0], e[1], e[2]);
      }
    }
    // the next iteration's first barrier orders these reads before the buffers are reused
  }
}

struct Config {
  int threads, ctas_per_sm;
  const void* fn;
};

const Config kConfigs[] = {
    {256, 2, reinterpret_cast<const void*>(&sweep_fp64_kernel<256, 2>)},
    {128, 4, reinterpret_cast<const void*>(&sweep_fp64_kernel<128, 4>)},
};

}  // namespace

cudaError_t launch_sweep_fp64_implicit(int cfg, const RomDev* objs, const SweepTask* table, int n_tasks,
                                       int* counter, const double* omega, int omega_stride, double* R,
                                       double* I, double* Delta, int* status, int n_w, int grid,
                                       size_t smem_bytes, double2* workspace, size_t ws_elems,
                                       cudaStream_t stream) {
  cudaError_t e;
  if (cfg == 0) {
    e = cudaFuncSetAttribute(sweep_fp64_kernel<256, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes);
    if (e != cudaSuccess) return e;
    sweep_fp64_kernel<256, 2, true><<<grid, 256, smem_bytes, stream>>>(
        objs, table, n_tasks, counter, omega, omega_stride, nullptr, R, I, Delta, nullptr, status, n_w, workspace,
        ws_elems);
  } else {
    e = cudaFuncSetAttribute(sweep_fp64_kernel<128, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes);
    if (e != cudaSuccess) return e;
    sweep_fp64_kernel<128, 4, true><<<grid, 128, smem_bytes, stream>>>(
        objs, table, n_tasks, counter, omega, omega_stride, nullptr, R, I, Delta, nullptr, status, n_w, workspace,
        ws_elems);
  }
  return cudaGetLastError();
}

cudaError_t launch_sweep_fp64_routed(int cfg, const RomDev* objs, const SweepTask* table, int* counter,
                                     const double* omega, int omega_stride, const double* s_sigma, double* R,
                                     double* I, double* Delta, double* eig, int* status, int n_w, int grid,
                                     size_t smem_bytes, double2* workspace, size_t ws_elems, cudaStream_t stream) {
  cudaError_t e;
  if (cfg == 0) {
    e = cudaFuncSetAttribute(sweep_fp64_kernel<256, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes);
    if (e != cudaSuccess) return e;
    sweep_fp64_kernel<256, 2, true><<<grid, 256, smem_bytes, stream>>>(
        objs, table, -1, counter, omega, omega_stride, s_sigma, R, I, Delta, eig, status, n_w, workspace, ws_elems);
  } else {
    e = cudaFuncSetAttribute(sweep_fp64_kernel<128, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes);
    if (e != cudaSuccess) return e;
    sweep_fp64_kernel<128, 4, true><<<grid, 128, smem_bytes, stream>>>(
        objs, table, -1, counter, omega, omega_stride, s_sigma, R, I, Delta, eig, status, n_w, workspace, ws_elems);
  }
  return cudaGetLastError();
}

int sweep_fp64_num_configs() { return (int)(sizeof(kConfigs) / sizeof(kConfigs[0])); }
int sweep_fp64_threads(int cfg) { return kConfigs[cfg].threads; }
int sweep_fp64_ctas_per_sm(int cfg) { return kConfigs[cfg].ctas_per_sm; }
const void* sweep_fp64_symbol(int cfg) { return kConfigs[cfg].fn; }
const void* sweep_fp64_implicit_symbol(int cfg) {
  return cfg == 0 ? (const void*)sweep_fp64_kernel<256, 2, true> : (const void*)sweep_fp64_kernel<128, 4, true>;
}

size_t sweep_fp64_matrix_elems(int r) { return (size_t)matrix_elems(r); }

size_t sweep_fp64_bytes_per_system(int r, bool matrix_in_smem) {
  const size_t am = matrix_in_smem ? sweep_fp64_matrix_elems(r) : 0;
  return 16 * (am + 3 * (size_t)r + (size_t)r) + 8 * (1 + (size_t)kRed * kSplit);
}

cudaError_t sweep_fp64_configure(int cfg, size_t smem_bytes) {
  return cudaFuncSetAttribute(kConfigs[cfg].fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

cudaError_t launch_sweep_fp64(int cfg, const RomDev* objs, const SweepTask* tasks, int n_tasks, int* counter,
                              const double* omega, int omega_stride, const double* s_sigma,
                              double* R, double* I, double* Delta, double* eig, int* status, int n_w, int grid,
                              size_t smem_bytes, double2* workspace, size_t ws_elems, cudaStream_t stream) {
  if (cfg == 0)
    sweep_fp64_kernel<256, 2><<<grid, 256, smem_bytes, stream>>>(objs, tasks, n_tasks, counter, omega,
                                                                omega_stride, s_sigma, R, I, Delta, eig, status,
                                                                n_w, workspace, ws_elems);
  else
    sweep_fp64_kernel<128, 4><<<grid, 128, smem_bytes, stream>>>(objs, tasks, n_tasks, counter, omega,
                                                                omega_stride, s_sigma, R, I, Delta, eig, status,
                                                                n_w, workspace, ws_elems);
  return cudaGetLastError();
}

}  // namespace mrom

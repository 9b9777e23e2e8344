// Vector-Jacobian product of the batched sweep (R, I) with respect to the frequency
// omega, a conductivity scale s_sigma and a permeability scale s_mu.
//
// Forward model per (object, omega) (Eqs. (17)-(19) with the scales applied):
//   w' = s_sigma omega,  K(s_mu) = K + (1/s_mu - 1) K_in,
//   A = K(s_mu) + Me - i w' C,  A P = i w' B,
//   R = -a^3/4 Re(P^H K(s_mu) P) (+ N0),  I = w' a^3/4 (c00 + Re(P^H C P + B^H P + P^H B)).
// For L = sum gR_ij R_ij + gI_ij I_ij, dL = Re tr(dP^H Z) with
//   Z = -a^3/4 K(s_mu) P G_R + w' a^3/4 (C P + B) G_I,   G = g + g^T,
// and with the adjoint Lambda = A^-H Z (same LU factors: U^H then L^H),
//   dL/domega = s_sigma Im tr((B + C P)^H Lambda) + sum gI_ij I_ij / omega,
//   dL/ds_mu  = (Re tr((K_in P)^H Lambda) + a^3/4 sum gR_ij Re(p_i^H K_in p_j)) / s_mu^2,
//   dL/ds_sigma = sum_omega (omega / s_sigma) dL/domega      (I(omega; s_sigma) = I(s_sigma omega; 1)).
// With the PODP in mu_r, B, c00 and N0 depend on s_mu as well (dB, dc00, dN0 per object), adding
//   Re tr(dB^H (w' a^3/4 P G_I - i w' Lambda)) + w' a^3/4 sum gI_ij dc00_ij + sum gR_ij dN0_ij
// to dL/ds_mu (P is linear in B through A P = i w' B, and I holds B directly).
// The factors are recomputed here instead of being stored per frequency.  This is the LU
// route; the pencil route of the same product is pencil_vjp_kernel (pencil.cu).
#include "mrom_internal.h"

#include <algorithm>
#include <numeric>

namespace mrom {
namespace {

constexpr int kT = 128;  // threads per CTA (4 CTAs per SM)
constexpr int kW = kT / 32;
constexpr int kRedV = 48;

__device__ __forceinline__ double2 c_msub(double2 c, double2 a, double2 b) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 c_conj_mac(double2 c, double2 a, double2 b) {  // c + conj(a) b
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 c_conj_msub(double2 c, double2 a, double2 b) {  // c - conj(a) b
  return make_double2(fma(-a.x, b.x, fma(-a.y, b.y, c.x)), fma(-a.x, b.y, fma(a.y, b.x, c.y)));
}
__device__ __forceinline__ double2 c_recip(double2 a, int* status) {
  const double d = fma(a.x, a.x, a.y * a.y);
  if (!(d > 0.0) || !isfinite(d)) {
    atomicOr(status, kStatusSingular);
    return make_double2(__longlong_as_double(0x7ff8000000000000LL), 0.0);
  }
  const double id = 1.0 / d;
  return make_double2(a.x * id, -a.y * id);
}

// Task t of a routed table (header entry 0: .obj = entries, .w0 = total tasks; then {object,
// frequencies per task, first task index, flags}).
__device__ __forceinline__ SweepTask routed_task(const SweepTask* __restrict__ table, int n_w, int t) {
  const int n = table[0].obj;
  int lo = 1, hi = n + 1;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (table[mid].w0 <= t) lo = mid; else hi = mid;
  }
  const SweepTask e = table[lo];
  const int w0 = (t - e.w0) * e.nw;
  return SweepTask{e.obj, w0, min(e.nw, n_w - w0), e.pad};
}

template <bool ROUTED>
__global__ void __launch_bounds__(kT, 4)
sweep_vjp_kernel(const VjpDev* __restrict__ objs, const SweepTask* __restrict__ tasks, int n_tasks,
                 int* __restrict__ counter, const double* __restrict__ omega, int omega_stride,
                 const double* __restrict__ s_sigma, const double* __restrict__ s_mu,
                 const double* __restrict__ gR, const double* __restrict__ gI, double* __restrict__ g_omega,
                 double* __restrict__ g_mu_part, double* __restrict__ Rout, double* __restrict__ Iout,
                 int* __restrict__ status, int n_w, double2* __restrict__ workspace, size_t ws_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_task;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (ROUTED) n_tasks = tasks[0].w0;
  for (;;) {
    if (tid == 0) s_task = atomicAdd(counter, 1);
    __syncthreads();
    const int t = s_task;
    __syncthreads();
    if (t >= n_tasks) break;
    const SweepTask task = ROUTED ? routed_task(tasks, n_w, t) : tasks[t];
    const VjpDev& ob = objs[task.obj];
    const int r = ob.r, S = task.nw, ld = r + 3;
    const size_t per_elems = (size_t)r * ld + 9 * (size_t)r;  // augmented system + y^K, y^C, y^Kin
    double2* sp = reinterpret_cast<double2*>(smem_raw);
    double2* Am;
    if (task.pad & 1) {
      Am = workspace + (size_t)blockIdx.x * ws_elems;
    } else {
      Am = sp;
      sp += (size_t)S * per_elems;
    }
    double2* Pm = sp;                                   // S * r * 3
    double2* Inv = Pm + (size_t)S * r * 3;              // S * r
    double* Ws = reinterpret_cast<double*>(Inv + (size_t)S * r);  // S
    double* Gs = Ws + S;                                // S * 18: symmetrised gR, gI
    double* Red = Gs + (size_t)S * 18;                  // S * kRedV
    const double ssig = s_sigma ? s_sigma[task.obj] : 1.0;
    const double smu = s_mu ? s_mu[task.obj] : 1.0;
    const double fmu = 1.0 / smu - 1.0;
    const bool kin = ob.Kin != nullptr;

    for (int s = tid; s < S; s += kT) {
      const double w = omega[(size_t)task.obj * omega_stride + task.w0 + s] * ssig;
      const bool ok = (w > 0.0) && isfinite(w) && (smu > 0.0) && (ssig > 0.0);
      if (!ok) atomicOr(status, kStatusBadOmega);
      Ws[s] = ok ? w : __longlong_as_double(0x7ff8000000000000LL);
    }
    for (int idx = tid; idx < S * 18; idx += kT) {
      const int s = idx / 18, q = idx % 18;
      const size_t e = ((size_t)task.obj * n_w + task.w0 + s) * 9;
      const double* g = q < 9 ? gR : gI;
      const int ij = q % 9, i = ij / 3, j = ij % 3;
      Gs[idx] = g[e + i * 3 + j] + g[e + j * 3 + i];
    }
    __syncthreads();

    // ---- forward: [K(s_mu) + Me - i w' C | i w' B], elimination, back substitution
    for (int idx = tid; idx < S * r * ld; idx += kT) {
      const int s = idx / (r * ld);
      const int e = idx - s * r * ld;
      const int i = e / ld, j = e - (e / ld) * ld;
      const double w = Ws[s];
      double2 v;
      if (j < r) {
        double2 k = ob.K[i * r + j];
        if (kin) {
          const double2 q = ob.Kin[i * r + j];
          k.x = fma(fmu, q.x, k.x);
          k.y = fma(fmu, q.y, k.y);
        }
        if (ob.Me) {
          const double2 m = ob.Me[i * r + j];
          k.x += m.x;
          k.y += m.y;
        }
        const double2 c = ob.C[i * r + j];
        v = make_double2(fma(w, c.y, k.x), fma(-w, c.x, k.y));
      } else {
        const double2 b = ob.B[i * 3 + (j - r)];
        v = make_double2(-w * b.y, w * b.x);
      }
      Am[(size_t)s * per_elems + e] = v;
      if (e == 0) Inv[(size_t)s * r] = c_recip(v, status);
    }
    __syncthreads();
    for (int k = 0; k < r - 1; ++k) {
      const int m = r - k - 1;
      for (int idx = tid; idx < S * m; idx += kT) {
        const int s = idx / m, i = k + 1 + (idx - (idx / m) * m);
        double2* a = Am + (size_t)s * per_elems;
        a[i * ld + k] = c_mul(a[i * ld + k], Inv[(size_t)s * r + k]);
      }
      __syncthreads();
      const int nc = ld - k - 1, per = m * nc;
      for (int idx = tid; idx < S * per; idx += kT) {
        const int s = idx / per, e = idx - (idx / per) * per;
        const int i = k + 1 + e / nc, j = k + 1 + (e - (e / nc) * nc);
        double2* a = Am + (size_t)s * per_elems;
        const double2 v = c_msub(a[i * ld + j], a[i * ld + k], a[k * ld + j]);
        a[i * ld + j] = v;
        if (e == 0) Inv[(size_t)s * r + k + 1] = c_recip(v, status);
      }
      __syncthreads();
    }
    for (int sj = warp; sj < S * 3; sj += kW) {
      const int s = sj / 3, j = sj - (sj / 3) * 3;
      double2* a = Am + (size_t)s * per_elems;
      const double2* inv = Inv + (size_t)s * r;
      double2* p = Pm + (size_t)s * r * 3;
      for (int k = r - 1; k >= 0; --k) {
        const double2 x = c_mul(a[k * ld + r + j], inv[k]);
        for (int i = lane; i < k; i += 32) a[i * ld + r + j] = c_msub(a[i * ld + r + j], a[i * ld + k], x);
        if (lane == 0) p[k * 3 + j] = x;
        __syncwarp();
      }
    }
    __syncthreads();

    // ---- y = M p for M in {K(s_mu), C, K_in} (Hermitian: M[a][b] = conj(M[b][a]), read along a)
    const int nmat = kin ? 3 : 2;
    for (int idx = tid; idx < S * nmat * r * 3; idx += kT) {
      const int s = idx / (nmat * r * 3);
      int e = idx - s * nmat * r * 3;
      const int mm = e / (r * 3);
      e -= mm * r * 3;
      const int a = e / 3, j = e - (e / 3) * 3;
      const double2* p = Pm + (size_t)s * r * 3;
      double2 y = make_double2(0.0, 0.0);
      for (int b = 0; b < r; ++b) {
        double2 g;
        if (mm == 0) {
          g = ob.K[b * r + a];
          if (kin) {
            const double2 q = ob.Kin[b * r + a];
            g.x = fma(fmu, q.x, g.x);
            g.y = fma(fmu, q.y, g.y);
          }
        } else {
          g = (mm == 1 ? ob.C : ob.Kin)[b * r + a];
        }
        y = c_conj_mac(y, g, p[b * 3 + j]);
      }
      Am[(size_t)s * per_elems + (size_t)r * ld + (mm * r + a) * 3 + j] = y;
    }
    __syncthreads();

    // ---- forward reductions: q 0..8 Re(p_i^H y^K_j), 9..17 Re(p_i^H y^C_j), 18..26 Re(b_i^H p_j),
    // 27..35 Re(p_i^H y^Kin_j); and the adjoint source Z in the right-hand-side columns
    for (int idx = tid; idx < S * 36; idx += kT) {
      const int s = idx / 36, q = idx % 36;
      if (q >= 27 && !kin) {
        Red[(size_t)s * kRedV + q] = 0.0;
        continue;
      }
      const int ij = q % 9, i = ij / 3, j = ij % 3;
      const double2* p = Pm + (size_t)s * r * 3;
      const double2* y = Am + (size_t)s * per_elems + (size_t)r * ld;
      double acc = 0.0;
      for (int a = 0; a < r; ++a) {
        if (q < 18 || q >= 27) {
          const int mm = q < 9 ? 0 : (q < 18 ? 1 : 2);
          const double2 pa = p[a * 3 + i], ya = y[(mm * r + a) * 3 + j];
          acc = fma(pa.x, ya.x, fma(pa.y, ya.y, acc));
        } else {
          const double2 b = ob.B[a * 3 + i], pa = p[a * 3 + j];
          acc = fma(b.x, pa.x, fma(b.y, pa.y, acc));
        }
      }
      Red[(size_t)s * kRedV + q] = acc;
    }
    for (int idx = tid; idx < S * r * 3; idx += kT) {
      const int s = idx / (r * 3), e = idx - (idx / (r * 3)) * (r * 3);
      const int a = e / 3, k = e - (e / 3) * 3;
      const double2* y = Am + (size_t)s * per_elems + (size_t)r * ld;
      const double* g = Gs + (size_t)s * 18;
      const double cR = -0.25 * ob.alpha3, cI = 0.25 * ob.alpha3 * Ws[s];
      double2 z = make_double2(0.0, 0.0);
      for (int j = 0; j < 3; ++j) {
        const double gr = cR * g[j * 3 + k], gi = cI * g[9 + j * 3 + k];
        const double2 yk = y[(0 * r + a) * 3 + j], yc = y[(1 * r + a) * 3 + j], b = ob.B[a * 3 + j];
        z.x = fma(gr, yk.x, fma(gi, yc.x + b.x, z.x));
        z.y = fma(gr, yk.y, fma(gi, yc.y + b.y, z.y));
      }
      Am[(size_t)s * per_elems + a * ld + r + k] = z;
    }
    __syncthreads();

    // ---- adjoint solves A^H Lambda = Z with A = L U: U^H w = Z (forward), L^H Lambda = w (backward)
    for (int sk = warp; sk < S * 3; sk += kW) {
      const int s = sk / 3, k3 = sk - (sk / 3) * 3;
      double2* a = Am + (size_t)s * per_elems;
      const double2* inv = Inv + (size_t)s * r;
      for (int k = 0; k < r; ++k) {
        const double2 iv = make_double2(inv[k].x, -inv[k].y);  // 1 / conj(u_kk)
        const double2 x = c_mul(a[k * ld + r + k3], iv);
        for (int i = k + 1 + lane; i < r; i += 32) a[i * ld + r + k3] = c_conj_msub(a[i * ld + r + k3], a[k * ld + i], x);
        __syncwarp();
        if (lane == 0) a[k * ld + r + k3] = x;
        __syncwarp();
      }
      for (int k = r - 1; k >= 0; --k) {
        const double2 x = a[k * ld + r + k3];
        for (int i = lane; i < k; i += 32) a[i * ld + r + k3] = c_conj_msub(a[i * ld + r + k3], a[k * ld + i], x);
        __syncwarp();
      }
    }
    __syncthreads();

    // ---- adjoint reductions: q 36: Im tr((B + C P)^H Lambda), q 37: Re tr((K_in P)^H Lambda);
    // with dB: q 38..46 Re(db_i^H p_j), q 47 Im tr(dB^H Lambda)
    const int nq_adj = ob.dB ? 12 : 2;
    for (int idx = tid; idx < S * nq_adj; idx += kT) {
      const int s = idx / nq_adj, q = idx % nq_adj;
      const double2* a = Am + (size_t)s * per_elems;
      const double2* y = a + (size_t)r * ld;
      double acc = 0.0;
      if (q >= 2 && q < 11) {
        const int i = (q - 2) / 3, j = (q - 2) % 3;
        const double2* p = Pm + (size_t)s * r * 3;
        for (int aa = 0; aa < r; ++aa) {
          const double2 db = ob.dB[aa * 3 + i], pa = p[aa * 3 + j];
          acc = fma(db.x, pa.x, fma(db.y, pa.y, acc));
        }
      } else if (q == 11) {
        for (int e = 0; e < r * 3; ++e) {
          const double2 lam = a[(e / 3) * ld + r + e % 3], db = ob.dB[e];
          acc += db.x * lam.y - db.y * lam.x;  // Im(conj(db) lam)
        }
      } else if (q == 0) {
        for (int e = 0; e < r * 3; ++e) {
          const int aa = e / 3, k = e % 3;
          const double2 lam = a[aa * ld + r + k], yc = y[(1 * r + aa) * 3 + k], b = ob.B[aa * 3 + k];
          const double2 v = make_double2(yc.x + b.x, yc.y + b.y);
          acc += v.x * lam.y - v.y * lam.x;  // Im(conj(v) lam)
        }
      } else if (kin) {
        for (int e = 0; e < r * 3; ++e) {
          const int aa = e / 3, k = e % 3;
          const double2 lam = a[aa * ld + r + k], yk = y[(2 * r + aa) * 3 + k];
          acc += yk.x * lam.x + yk.y * lam.y;
        }
      }
      Red[(size_t)s * kRedV + 36 + q] = acc;
    }
    __syncthreads();

    // ---- outputs
    for (int s = tid; s < S; s += kT) {
      const double* red = Red + (size_t)s * kRedV;
      const double* g = Gs + (size_t)s * 18;
      const double w = Ws[s];
      const size_t o = (size_t)task.obj * n_w + task.w0 + s;
      double gI_dot_I = 0.0, gR_dot_HKin = 0.0;
      for (int ij = 0; ij < 9; ++ij) {
        const int i = ij / 3, j = ij % 3, ji = j * 3 + i;
        const double Rv = -0.25 * ob.alpha3 * 0.5 * (red[ij] + red[ji]) + ob.N0[ij];
        const double Iv = 0.25 * ob.alpha3 * w * (ob.c00[ij] + 0.5 * (red[9 + ij] + red[9 + ji]) + red[18 + ij] + red[18 + ji]);
        if (Rout) Rout[o * 9 + ij] = Rv;
        if (Iout) Iout[o * 9 + ij] = Iv;
        // g holds gR + gR^T and gI + gI^T; the sums over all (i, j) count each pair twice
        gI_dot_I += 0.5 * g[9 + ij] * Iv;
        gR_dot_HKin += 0.5 * g[ij] * 0.5 * (red[27 + ij] + red[27 + ji]);
      }
      const double wr = w / ssig;  // the caller's omega
      g_omega[o] = ssig * red[36] + gI_dot_I / wr;
      double gmu = (red[37] + 0.25 * ob.alpha3 * gR_dot_HKin) / (smu * smu);
      if (ob.dB) {
        double src = 0.0, stat = 0.0;
        for (int ij = 0; ij < 9; ++ij) {
          src = fma(red[38 + ij], g[9 + ij], src);
          stat = fma(0.5 * g[9 + ij], 0.25 * ob.alpha3 * w * ob.dc00[ij], fma(0.5 * g[ij], ob.dN0[ij], stat));
        }
        gmu += 0.25 * ob.alpha3 * w * src + w * red[47] + stat;
      }
      g_mu_part[o] = gmu;
    }
  }
}

// per object: g_ssigma = sum_w (omega_w / s_sigma) g_omega, g_smu = sum_w parts (fixed order)
__global__ void vjp_object_sums_kernel(const double* __restrict__ omega, int omega_stride, const double* __restrict__ s_sigma,
                                       const double* __restrict__ g_omega, const double* __restrict__ g_mu_part, int n_obj,
                                       int n_w, double* __restrict__ g_ssigma, double* __restrict__ g_smu) {
  const int o = blockIdx.x;
  __shared__ double a[256], b[256];
  double sa = 0.0, sb = 0.0;
  const double ss = s_sigma ? s_sigma[o] : 1.0;
  for (int k = threadIdx.x; k < n_w; k += blockDim.x) {
    const size_t e = (size_t)o * n_w + k;
    sa += omega[(size_t)o * omega_stride + k] / ss * g_omega[e];
    sb += g_mu_part[e];
  }
  a[threadIdx.x] = sa;
  b[threadIdx.x] = sb;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      a[threadIdx.x] += a[threadIdx.x + s];
      b[threadIdx.x] += b[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (g_ssigma) g_ssigma[o] = a[0];
    if (g_smu) g_smu[o] = b[0];
  }
}

size_t vjp_bytes_per_system(int r, bool in_smem) {
  const size_t am = in_smem ? (size_t)r * (r + 3) + 9 * (size_t)r : 0;
  return 16 * (am + 3 * (size_t)r + (size_t)r) + 8 * (1 + 18 + kRedV);
}

}  // namespace
}  // namespace mrom

using namespace mrom;

extern "C" mrom_status mrom_sweep_vjp(mrom_handle h, const mrom_rom_t* roms, int32_t n_obj, const double* omega,
                                      int32_t n_w, int32_t omega_stride, const double* s_sigma, const double* s_mu,
                                      const double* gR, const double* gI, double* g_omega, double* g_ssigma,
                                      double* g_smu, double* R, double* I) {
  if (!h) return MROM_EINVAL;
  if (!roms || n_obj < 1 || n_w < 1 || !omega || !gR || !gI || !g_omega)
    return fail(h, MROM_EINVAL, "mrom_sweep_vjp: bad arguments");
  if (omega_stride != 0 && omega_stride < n_w)
    return fail(h, MROM_EINVAL, "mrom_sweep_vjp: omega_stride must be 0 or >= n_w");
  for (int o = 0; o < n_obj; ++o) {
    if (!roms[o] || roms[o]->ctx != h) return fail(h, MROM_EINVAL, "mrom_sweep_vjp: invalid object");
    if (roms[o]->r_dirs[0] + roms[o]->r_dirs[1] + roms[o]->r_dirs[2] > 0)
      return fail(h, MROM_ENOTSUP, "mrom_sweep_vjp: objects with one basis per direction are swept by mrom_sweep");
    if ((s_mu || g_smu) && !roms[o]->has_kin)
      return fail(h, MROM_EINVAL, "mrom_sweep_vjp: s_mu / g_smu need K_in on every object");
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep_vjp: cudaSetDevice");
  int per_sm = 0;
  cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
  const size_t budget = std::min<size_t>(h->smem_optin, (size_t)per_sm / 4) - 2048;
  std::vector<VjpDev> objs(n_obj);
  std::vector<SweepTask> tasks;
  std::vector<double> cost;
  std::vector<int2> lu_shape(n_obj);
  size_t smem = 0, ws_elems = 0;
  int64_t n_tasks_all = 0;
  const bool pencil = h->solver == MROM_SOLVER_AUTO;  // every object here has one shared basis
  for (int o = 0; o < n_obj; ++o) {
    const mrom_rom* m = roms[o];
    VjpDev& d = objs[o];
    d.K = m->K;
    d.Kin = m->has_kin ? m->Kin : nullptr;
    d.C = m->C;
    d.Me = m->Me;
    d.B = m->B;
    std::copy(m->c00, m->c00 + 9, d.c00);
    std::copy(m->N0, m->N0 + 9, d.N0);
    d.alpha3 = m->alpha * m->alpha * m->alpha;
    d.r = m->r;
    const size_t per_s = vjp_bytes_per_system(m->r, true);
    const bool in_smem = per_s <= budget;
    const size_t per = in_smem ? per_s : vjp_bytes_per_system(m->r, false);
    const int S = in_smem ? std::min<int>(n_w, (int)(budget / per_s)) : 1;
    if (!in_smem) ws_elems = std::max(ws_elems, (size_t)m->r * (m->r + 3) + 9 * (size_t)m->r);
    smem = std::max(smem, per * std::min(S, n_w));
    n_tasks_all += (n_w + S - 1) / S;
    lu_shape[o] = make_int2(S, in_smem ? 0 : 1);
    if (pencil) continue;  // the LU kernel runs over the device-routed table
    const double r = m->r;
    for (int w0 = 0; w0 < n_w; w0 += S) {
      const int nw = std::min(S, n_w - w0);
      tasks.push_back(SweepTask{o, w0, nw, in_smem ? 0 : 1});
      cost.push_back((8.0 * r * r * r / 3.0 + 40.0 * r * r) * nw);
    }
  }
  // PODP in mu_r: objects with a reduced static problem get B(s_mu) (and dB/ds_mu when the
  // permeability gradient is wanted) in per-call buffers, filled on the device below
  const bool deriv = g_smu != nullptr;
  std::vector<MuDev> mus(n_obj);
  size_t mu_elems = 0;
  int m_max = 0;
  for (int o = 0; o < n_obj; ++o) {
    if (roms[o]->mu.m > 0) {
      mu_elems += (deriv ? 6 : 3) * (size_t)roms[o]->r;
      m_max = std::max(m_max, roms[o]->mu.m);
    }
  }
  void* mublk = nullptr;
  MuDev* d_mus = nullptr;
  if (m_max > 0) {
    const size_t b_mus = (n_obj * sizeof(MuDev) + 255) / 256 * 256;
    e = cudaMallocAsync(&mublk, b_mus + mu_elems * sizeof(double2), h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep_vjp: allocation");
    d_mus = static_cast<MuDev*>(mublk);
    auto* q = reinterpret_cast<double2*>(static_cast<char*>(mublk) + b_mus);
    for (int o = 0; o < n_obj; ++o) {
      if (roms[o]->mu.m <= 0) continue;
      const int r = roms[o]->r;
      mus[o] = roms[o]->mu;
      mus[o].Bdst = q; q += 3 * (size_t)r;
      mus[o].dBdst = deriv ? q : nullptr;
      if (deriv) q += 3 * (size_t)r;
      objs[o].B = mus[o].Bdst;
      objs[o].dB = mus[o].dBdst;
    }
    e = cudaMemcpyAsync(d_mus, mus.data(), n_obj * sizeof(MuDev), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) {
      cudaFreeAsync(mublk, h->stream);
      return cuda_fail(h, e, "mrom_sweep_vjp: upload");
    }
  }
  // pencil route: tables (V^H K_in V when the permeability gradient is wanted), then
  // preparation and routing on the device
  PencilTables pt;
  std::vector<RomDev> recs;
  if (pencil) {
    recs.resize(n_obj);
    for (int o = 0; o < n_obj; ++o) {
      recs[o] = rom_record(roms[o]);
      if (roms[o]->mu.m > 0) {
        recs[o].B = mus[o].Bdst;
        recs[o].dB = mus[o].dBdst;
      }
    }
    std::vector<int> order_lu(n_obj);
    std::iota(order_lu.begin(), order_lu.end(), 0);
    std::stable_sort(order_lu.begin(), order_lu.end(), [&](int a, int b) { return recs[a].r > recs[b].r; });
    std::vector<int2> lu_info(n_obj);
    for (int k = 0; k < n_obj; ++k) lu_info[k] = lu_shape[order_lu[k]];
    const mrom_status ps = pencil_tables_create(h, recs, n_w, false, g_smu != nullptr, order_lu, lu_info, &pt);
    if (ps != MROM_OK) {
      if (mublk) cudaFreeAsync(mublk, h->stream);
      return ps;
    }
  }
  std::vector<int> order(tasks.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<SweepTask> sorted(tasks.size());
  for (size_t k = 0; k < order.size(); ++k) sorted[k] = tasks[order[k]];
  const void* lu_fn = pencil ? reinterpret_cast<const void*>(&sweep_vjp_kernel<true>)
                             : reinterpret_cast<const void*>(&sweep_vjp_kernel<false>);
  e = cudaFuncSetAttribute(lu_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lu_fn, kT, smem);
  if (e != cudaSuccess) {
    pencil_tables_destroy(&pt, h->stream);
    if (mublk) cudaFreeAsync(mublk, h->stream);
    return cuda_fail(h, e, "mrom_sweep_vjp: configuration");
  }
  const int grid = (int)std::min<int64_t>(n_tasks_all, (int64_t)h->num_sms * std::max(occ, 1));
  const size_t ws_bytes = ws_elems * sizeof(double2) * grid;
  const size_t b_recs = pencil ? (n_obj * sizeof(RomDev) + 255) / 256 * 256 : 0;
  const size_t bytes = ws_bytes + (size_t)n_obj * n_w * sizeof(double) + n_obj * sizeof(VjpDev) +
                       sorted.size() * sizeof(SweepTask) + 16 + b_recs + 256;
  void* blk = nullptr;
  e = cudaMallocAsync(&blk, bytes, h->stream);
  if (e != cudaSuccess) {
    pencil_tables_destroy(&pt, h->stream);
    if (mublk) cudaFreeAsync(mublk, h->stream);
    return cuda_fail(h, e, "mrom_sweep_vjp: allocation");
  }
  char* p = static_cast<char*>(blk);
  auto* d_ws = ws_elems ? reinterpret_cast<double2*>(p) : nullptr;
  p += ws_bytes;
  auto* d_gmu = reinterpret_cast<double*>(p);
  p += (size_t)n_obj * n_w * sizeof(double);
  auto* d_recs = reinterpret_cast<RomDev*>(p);
  p += b_recs;
  auto* d_objs = reinterpret_cast<VjpDev*>(p);
  p += n_obj * sizeof(VjpDev);
  auto* d_tasks = reinterpret_cast<SweepTask*>(p);
  p += sorted.size() * sizeof(SweepTask);
  auto* d_counter = reinterpret_cast<int*>(p);
  e = cudaMemcpyAsync(d_objs, objs.data(), n_obj * sizeof(VjpDev), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && !pencil)
    e = cudaMemcpyAsync(d_tasks, sorted.data(), sorted.size() * sizeof(SweepTask), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_counter, 0, sizeof(int), h->stream);
  if (e == cudaSuccess && pencil)
    e = cudaMemcpyAsync(d_recs, recs.data(), n_obj * sizeof(RomDev), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && d_mus) {  // B, c00, N0 (and derivatives) at each object's s_mu
    e = launch_mu_instance(d_mus, n_obj, m_max, s_mu, deriv, pencil ? d_recs : nullptr, d_objs, h->d_status,
                           h->stream);
    ++h->launches;
  }
  if (e == cudaSuccess && pencil) {
    if (e == cudaSuccess) e = pencil_tables_prepare(h, pt, d_recs, omega, omega_stride, s_sigma, s_mu);
    if (e == cudaSuccess) e = pencil_tables_route(h, pt);
    if (e == cudaSuccess)
      e = launch_pencil_vjp(d_recs, pt.d_pens, pt.d_table_pen, pt.d_counters + 2, omega, omega_stride, s_sigma, s_mu,
                            gR, gI, g_omega, d_gmu, R, I, h->d_status, n_w, pt.pen_grid, pt.pen_smem_vjp, h->stream);
    if (e == cudaSuccess) {
      ++h->launches;
      sweep_vjp_kernel<true><<<grid, kT, smem, h->stream>>>(d_objs, pt.d_table_lu, -1, pt.d_counters + 3, omega,
                                                            omega_stride, s_sigma, s_mu, gR, gI, g_omega, d_gmu, R, I,
                                                            h->d_status, n_w, d_ws, ws_elems);
      e = cudaGetLastError();
    }
  } else if (e == cudaSuccess) {
    sweep_vjp_kernel<false><<<grid, kT, smem, h->stream>>>(d_objs, d_tasks, (int)sorted.size(), d_counter, omega,
                                                           omega_stride, s_sigma, s_mu, gR, gI, g_omega, d_gmu, R, I,
                                                           h->d_status, n_w, d_ws, ws_elems);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && (g_ssigma || g_smu)) {
    vjp_object_sums_kernel<<<n_obj, 256, 0, h->stream>>>(omega, omega_stride, s_sigma, g_omega, d_gmu, n_obj, n_w,
                                                         g_ssigma, g_smu);
    e = cudaGetLastError();
    ++h->launches;
  }
  cudaFreeAsync(blk, h->stream);
  pencil_tables_destroy(&pt, h->stream);
  if (mublk) cudaFreeAsync(mublk, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_sweep_vjp: launch");
  ++h->launches;
  return MROM_OK;
}

// PODP in the relative permeability: the reduced static problem of an object, instantiated
// per call at its permeability scale s (mu_r -> s mu_r on the object).
//
// Sect. 4.2 notes that the precomputation of Eqs. (17)-(19) carries over to parameters other
// than omega.  For mu_r the stiffness is affine in 1/s (Eq. (10a) is linear in mu_r^-1 cell by
// cell), and theta~^(0), which enters b, c00 and N0 (Eq. (6a)), solves a static problem whose
// operator depends on s; that problem is reduced by a POD basis V of static snapshots:
//   S(s) y = -(kout + kin / s),  S(s) = Sout + Sin / s + Mv   (m x m Hermitian positive definite)
//   B(s)   = Bx + BV y
//   c00(s) = cxx + Re(cvx^H y + y^H cvx + y^H cvv y)
//   N0(s)  = (nB - mB / s) I + a^3/4 Re(y^H (Sout + Sin / s) y)
// and, for the permeability gradient, d/ds of each with S dy = (kin + Sin y) / s^2.
// One CTA per object; m <= MROM_MAX_STATIC, so S and the m x 3 blocks stay in shared memory.
#include "mrom_internal.h"

#include <algorithm>
#include <vector>

namespace mrom {
namespace {

constexpr int kMT = 128;

__device__ __forceinline__ double2 cfma(double2 c, double2 a, double2 b) {  // c + a b
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// Solve L L^H X = X in place for the m x 3 block X (row-major, stride 3); one thread per column.
__device__ void chol_solve3(const double2* __restrict__ L, int m, double2* __restrict__ X) {
  const int j = threadIdx.x;
  if (j < 3) {
    for (int i = 0; i < m; ++i) {  // L z = x
      double2 v = X[i * 3 + j];
      for (int k = 0; k < i; ++k) {
        const double2 l = L[i * m + k], z = X[k * 3 + j];
        v.x -= l.x * z.x - l.y * z.y;
        v.y -= l.x * z.y + l.y * z.x;
      }
      const double d = L[i * m + i].x;
      X[i * 3 + j] = make_double2(v.x / d, v.y / d);
    }
    for (int i = m - 1; i >= 0; --i) {  // L^H x = z
      double2 v = X[i * 3 + j];
      for (int k = i + 1; k < m; ++k) {
        const double2 l = L[k * m + i], z = X[k * 3 + j];  // conj(L[k][i]) z
        v.x -= l.x * z.x + l.y * z.y;
        v.y -= l.x * z.y - l.y * z.x;
      }
      const double d = L[i * m + i].x;
      X[i * 3 + j] = make_double2(v.x / d, v.y / d);
    }
  }
  __syncthreads();
}

// Y (m x 3) = M X for a Hermitian m x m matrix M (row-major, global) plus an optional second
// matrix scaled by c: Y = (M1 + c M2) X.
__device__ void hmat3(const double2* __restrict__ M1, const double2* __restrict__ M2, double c, int m,
                      const double2* __restrict__ X, double2* __restrict__ Y) {
  for (int idx = threadIdx.x; idx < 3 * m; idx += kMT) {
    const int a = idx / 3, j = idx - (idx / 3) * 3;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = 0; b < m; ++b) {
      double2 v = M1[a * m + b];
      if (M2) {
        const double2 w = M2[a * m + b];
        v.x = fma(c, w.x, v.x);
        v.y = fma(c, w.y, v.y);
      }
      acc = cfma(acc, v, X[b * 3 + j]);
    }
    Y[idx] = acc;
  }
}

// Re(u_i^H v_j) for m x 3 blocks u, v (column i of u, column j of v)
__device__ __forceinline__ double re_dot(const double2* __restrict__ u, const double2* __restrict__ v, int m, int i,
                                         int j) {
  double acc = 0.0;
  for (int a = 0; a < m; ++a) {
    const double2 x = u[a * 3 + i], y = v[a * 3 + j];
    acc = fma(x.x, y.x, fma(x.y, y.y, acc));
  }
  return acc;
}

__global__ void __launch_bounds__(kMT)
mu_instance_kernel(const MuDev* __restrict__ mus, const double* __restrict__ s_mu, int deriv,
                   RomDev* __restrict__ recs, VjpDev* __restrict__ vjp, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_bad;
  const int o = blockIdx.x, tid = threadIdx.x;
  const MuDev& mu = mus[o];
  const int m = mu.m, r = mu.r;
  if (m <= 0) return;
  const double s = s_mu ? s_mu[o] : 1.0;
  if (!(s > 0.0) || !isfinite(s)) {
    if (tid == 0) atomicOr(status, kStatusBadOmega);
    return;
  }
  const double is = 1.0 / s, is2 = is * is;
  double2* L = reinterpret_cast<double2*>(smem_raw);  // m x m
  double2* y = L + (size_t)m * m;                     // m x 3 each below
  double2* dy = y + 3 * m;
  double2* Cy = dy + 3 * m;   // cvv y
  double2* Ky = Cy + 3 * m;   // (Sout + Sin / s) y
  double2* Sy = Ky + 3 * m;   // Sin y
  double2* Cdy = Sy + 3 * m;  // cvv dy
  double2* Kdy = Cdy + 3 * m; // (Sout + Sin / s) dy
  if (tid == 0) s_bad = 0;
  for (int idx = tid; idx < m * m; idx += kMT) {
    const double2 a = mu.Sout[idx], b = mu.Sin[idx], c = mu.Mv[idx];
    L[idx] = make_double2(fma(is, b.x, a.x) + c.x, fma(is, b.y, a.y) + c.y);
  }
  for (int idx = tid; idx < 3 * m; idx += kMT) {
    const double2 a = mu.kout[idx], b = mu.kin[idx];
    y[idx] = make_double2(-fma(is, b.x, a.x), -fma(is, b.y, a.y));
  }
  __syncthreads();
  // Cholesky S = L L^H (lower triangle, right-looking)
  for (int k = 0; k < m; ++k) {
    if (tid == 0) {
      const double d = L[k * m + k].x;
      if (!(d > 0.0) || !isfinite(d)) s_bad = 1;
      L[k * m + k] = make_double2(sqrt(d > 0.0 ? d : 1.0), 0.0);
    }
    __syncthreads();
    const double inv = 1.0 / L[k * m + k].x;
    for (int i = k + 1 + tid; i < m; i += kMT) {
      const double2 v = L[i * m + k];
      L[i * m + k] = make_double2(v.x * inv, v.y * inv);
    }
    __syncthreads();
    const int n = m - k - 1;
    for (int idx = tid; idx < n * n; idx += kMT) {
      const int i = k + 1 + idx / n, j = k + 1 + idx % n;
      if (j > i) continue;
      const double2 a = L[i * m + k], b = L[j * m + k];  // L[i][j] -= a conj(b)
      double2 v = L[i * m + j];
      v.x -= a.x * b.x + a.y * b.y;
      v.y -= a.y * b.x - a.x * b.y;
      L[i * m + j] = v;
    }
    __syncthreads();
  }
  if (s_bad) {
    if (tid == 0) atomicOr(status, kStatusSingular);
    return;
  }
  chol_solve3(L, m, y);
  if (mu.ydst)
    for (int idx = tid; idx < 3 * m; idx += kMT) mu.ydst[idx] = y[idx];
  hmat3(mu.cvv, nullptr, 0.0, m, y, Cy);
  hmat3(mu.Sout, mu.Sin, is, m, y, Ky);
  hmat3(mu.Sin, nullptr, 0.0, m, y, Sy);
  __syncthreads();
  if (deriv) {
    for (int idx = tid; idx < 3 * m; idx += kMT) {
      const double2 a = mu.kin[idx], b = Sy[idx];
      dy[idx] = make_double2((a.x + b.x) * is2, (a.y + b.y) * is2);
    }
    __syncthreads();
    chol_solve3(L, m, dy);
    hmat3(mu.cvv, nullptr, 0.0, m, dy, Cdy);
    hmat3(mu.Sout, mu.Sin, is, m, dy, Kdy);
  }
  // B(s) = Bx + BV y and dB = BV dy (r x 3)
  for (int idx = tid; idx < 3 * r; idx += kMT) {
    const int a = idx / 3, j = idx - (idx / 3) * 3;
    double2 b = mu.Bx[idx], db = make_double2(0.0, 0.0);
    for (int k = 0; k < m; ++k) {
      const double2 v = mu.BV[a * m + k];
      b = cfma(b, v, y[k * 3 + j]);
      if (deriv) db = cfma(db, v, dy[k * 3 + j]);
    }
    mu.Bdst[idx] = b;
    if (deriv) mu.dBdst[idx] = db;
  }
  __syncthreads();
  // c00, N0 and their derivatives: one thread per (quantity, i, j)
  if (tid < (deriv ? 36 : 18)) {
    const int qn = tid / 9, ij = tid % 9, i = ij / 3, j = ij % 3;
    const double q4 = 0.25 * mu.alpha3;
    double v;
    if (qn == 0) {
      v = mu.cxx[ij] + re_dot(mu.cvx, y, m, i, j) + re_dot(y, mu.cvx, m, i, j) + re_dot(y, Cy, m, i, j);
    } else if (qn == 1) {
      v = (i == j ? mu.nB - mu.mB * is : 0.0) + q4 * re_dot(y, Ky, m, i, j);
    } else if (qn == 2) {
      v = re_dot(mu.cvx, dy, m, i, j) + re_dot(dy, mu.cvx, m, i, j) + re_dot(dy, Cy, m, i, j) +
          re_dot(y, Cdy, m, i, j);
    } else {
      v = (i == j ? mu.mB * is2 : 0.0) +
          q4 * (re_dot(dy, Ky, m, i, j) + re_dot(y, Kdy, m, i, j) - is2 * re_dot(y, Sy, m, i, j));
    }
    if (recs) {
      RomDev& d = recs[o];
      (qn == 0 ? d.c00 : qn == 1 ? d.N0 : qn == 2 ? d.dc00 : d.dN0)[ij] = v;
    }
    if (vjp) {
      VjpDev& d = vjp[o];
      (qn == 0 ? d.c00 : qn == 1 ? d.N0 : qn == 2 ? d.dc00 : d.dN0)[ij] = v;
    }
  }
}

// Certificate blocks at s from the extended Gram (indices: sources 0..2, V 3..3+m, K_out block
// O = 3+m, K_in block I = O+r, C block Cb = I+r; G[u][v] = phi_u^H X^-1 phi_v):
//   G_KK(s)[a][b] = G[O+a][O+b] + (G[O+a][I+b] + G[I+a][O+b]) / s + G[I+a][I+b] / s^2
//   G_CK(s) - G_KC(s) = G[Cb+a][O+b] + G[Cb+a][I+b] / s - G[O+a][Cb+b] - G[I+a][Cb+b] / s
//   g_sK(s)[i][a] = sum_u conj(T_ui) (G[u][O+a] + G[u][I+a] / s),  g_sC(s)[i][a] = sum_u conj(T_ui) G[u][Cb+a]
//   gss(s)[i][j] = Re sum_uv conj(T_ui) G[u][v] T_vj,  T = [I_3 ; y(s)] (the sources C o_i(s) = C x_i + C V y_i).
__global__ void __launch_bounds__(kMT)
mu_cert_kernel(const MuDev* __restrict__ mus, const double* __restrict__ s_mu, RomDev* __restrict__ recs) {
  const int o = blockIdx.x, tid = threadIdx.x;
  const MuDev& mu = mus[o];
  if (mu.m <= 0 || !mu.Gext || !mu.ydst) return;
  const double s = s_mu ? s_mu[o] : 1.0;
  if (!(s > 0.0) || !isfinite(s)) return;  // reported by the instance kernel
  const double is = 1.0 / s, is2 = is * is;
  const int m = mu.m, r = mu.r, n = mu.next;
  const int V0 = 3, O0 = 3 + m, I0 = O0 + r, C0 = I0 + r;
  const double2* G = mu.Gext;
  const double2* y = mu.ydst;
  auto g = [&](int u, int v) { return G[(size_t)u * n + v]; };
  for (int idx = tid; idx < r * r; idx += kMT) {
    const int a = idx / r, b = idx - (idx / r) * r;
    const double2 oo = g(O0 + a, O0 + b), oi = g(O0 + a, I0 + b), io = g(I0 + a, O0 + b), ii = g(I0 + a, I0 + b);
    mu.GKKdst[idx] = make_double2(oo.x + (oi.x + io.x) * is + ii.x * is2, oo.y + (oi.y + io.y) * is + ii.y * is2);
    const double2 co = g(C0 + a, O0 + b), ci = g(C0 + a, I0 + b), oc = g(O0 + a, C0 + b), ic = g(I0 + a, C0 + b);
    mu.GSkdst[idx] = make_double2(co.x + ci.x * is - oc.x - ic.x * is, co.y + ci.y * is - oc.y - ic.y * is);
  }
  // T_ui: 1 for u = i < 3, y[(u-3)*3 + i] for V rows
  for (int idx = tid; idx < 3 * r; idx += kMT) {
    const int i = idx / r, a = idx - (idx / r) * r;
    double2 k = g(i, O0 + a), ki = g(i, I0 + a), c = g(i, C0 + a);
    k.x += ki.x * is;
    k.y += ki.y * is;
    for (int q = 0; q < m; ++q) {
      const double2 t = y[q * 3 + i];  // conj(t) * G
      const double2 vo = g(V0 + q, O0 + a), vi = g(V0 + q, I0 + a), vc = g(V0 + q, C0 + a);
      const double2 vk = make_double2(vo.x + vi.x * is, vo.y + vi.y * is);
      k = cfma(k, make_double2(t.x, -t.y), vk);
      c = cfma(c, make_double2(t.x, -t.y), vc);
    }
    mu.gsKdst[idx] = k;
    mu.gsCdst[idx] = c;
  }
  if (tid < 9) {
    const int i = tid / 3, j = tid % 3;
    double2 acc = g(i, j);
    for (int q = 0; q < m; ++q) {
      const double2 yj = y[q * 3 + j], yi = y[q * 3 + i];
      acc = cfma(acc, g(i, V0 + q), yj);                                   // G[i][V] y_j
      acc = cfma(acc, make_double2(yi.x, -yi.y), g(V0 + q, j));            // conj(y_i) G[V][j]
      double2 row = make_double2(0.0, 0.0);
      for (int l = 0; l < m; ++l) row = cfma(row, g(V0 + q, V0 + l), y[l * 3 + j]);
      acc = cfma(acc, make_double2(yi.x, -yi.y), row);                     // conj(y_i) G[V][V] y_j
    }
    recs[o].gss[tid] = acc.x;
  }
}

__global__ void scale_k_kernel(const ScaleKJob* __restrict__ jobs, const double* __restrict__ s_mu) {
  const ScaleKJob j = jobs[blockIdx.y];
  if (!j.dst) return;
  const double f = (s_mu ? 1.0 / s_mu[blockIdx.y] : 1.0) - 1.0;
  const int rr = j.r * j.r;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < rr; idx += gridDim.x * blockDim.x) {
    const double2 k = j.K[idx], q = j.Kin[idx];
    j.dst[idx] = make_double2(fma(f, q.x, k.x), fma(f, q.y, k.y));
  }
}

}  // namespace

cudaError_t launch_mu_cert(const MuDev* mus, int n_obj, const double* s_mu, RomDev* recs, cudaStream_t stream) {
  if (n_obj <= 0) return cudaSuccess;
  mu_cert_kernel<<<n_obj, kMT, 0, stream>>>(mus, s_mu, recs);
  return cudaGetLastError();
}

cudaError_t launch_scale_k(const ScaleKJob* jobs, int n_obj, int rmax, const double* s_mu, cudaStream_t stream) {
  if (n_obj <= 0) return cudaSuccess;
  scale_k_kernel<<<dim3((unsigned)std::max(1, std::min(64, (rmax * rmax + 255) / 256)), (unsigned)n_obj), 256, 0,
                   stream>>>(jobs, s_mu);
  return cudaGetLastError();
}

size_t mu_instance_smem_bytes(int m_max) { return ((size_t)m_max * m_max + 24 * (size_t)m_max) * sizeof(double2); }

cudaError_t launch_mu_instance(const MuDev* mus, int n_obj, int m_max, const double* s_mu, bool deriv, RomDev* recs,
                               VjpDev* vjp, int* status, cudaStream_t stream) {
  if (n_obj <= 0 || m_max <= 0) return cudaSuccess;
  const size_t smem = mu_instance_smem_bytes(m_max);
  cudaError_t e = cudaFuncSetAttribute(mu_instance_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mu_instance_kernel<<<n_obj, kMT, smem, stream>>>(mus, s_mu, deriv ? 1 : 0, recs, vjp, status);
  return cudaGetLastError();
}

}  // namespace mrom

using namespace mrom;

extern "C" int32_t mrom_rom_static_rank(mrom_rom_t rom) { return rom ? rom->mu.m : 0; }

extern "C" mrom_status mrom_rom_mu_state(mrom_rom_t rom, double s_mu, void* B, double* c00, double* N0, void* dB,
                                         double* dc00, double* dN0) {
  if (!rom) return MROM_EINVAL;
  mrom_ctx* h = rom->ctx;
  if (rom->mu.m <= 0) return fail(h, MROM_EINVAL, "mrom_rom_mu_state: the object has no static reduction");
  if (!(s_mu > 0.0) || !std::isfinite(s_mu)) return fail(h, MROM_EINVAL, "mrom_rom_mu_state: s_mu must be > 0");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_rom_mu_state: cudaSetDevice");
  const int r = rom->r;
  DevBuf buf;
  const size_t nb = 6 * (size_t)r * sizeof(double2) + sizeof(MuDev) + sizeof(RomDev) + sizeof(double) + 64;
  e = cudaMalloc(&buf.p, nb);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_rom_mu_state: allocation");
  char* p = static_cast<char*>(buf.p);
  auto* dBs = reinterpret_cast<double2*>(p);
  auto* ddB = dBs + 3 * (size_t)r;
  auto* dmu = reinterpret_cast<MuDev*>(ddB + 3 * (size_t)r);
  auto* drec = reinterpret_cast<RomDev*>(dmu + 1);
  auto* ds = reinterpret_cast<double*>(drec + 1);
  MuDev mu = rom->mu;
  mu.Bdst = dBs;
  mu.dBdst = ddB;
  cudaStream_t st = h->stream;
  e = cudaMemcpyAsync(dmu, &mu, sizeof(MuDev), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ds, &s_mu, sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_mu_instance(dmu, 1, rom->mu.m, ds, true, drec, nullptr, h->d_status, st);
  RomDev rec{};
  std::vector<double2> hb(6 * (size_t)r);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), dBs, hb.size() * sizeof(double2), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&rec, drec, sizeof(RomDev), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_rom_mu_state");
  ++h->launches;
  const mrom_status ss = mrom_synchronize(h);
  if (ss != MROM_OK) return ss;
  if (B) std::copy(hb.begin(), hb.begin() + 3 * r, static_cast<double2*>(B));
  if (dB) std::copy(hb.begin() + 3 * r, hb.end(), static_cast<double2*>(dB));
  if (c00) std::copy(rec.c00, rec.c00 + 9, c00);
  if (N0) std::copy(rec.N0, rec.N0 + 9, N0);
  if (dc00) std::copy(rec.dc00, rec.dc00 + 9, dc00);
  if (dN0) std::copy(rec.dN0, rec.dN0 + 9, dN0);
  return MROM_OK;
}

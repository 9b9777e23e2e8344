// Rotation-invariant features of the spectral signature (Sect. 1): under a rotation Q of the
// object each coefficient matrix becomes Q M Q^T, so the eigenvalues of R~ = N0 + R and of I
// at each frequency are orientation independent and serve for dictionary matching.  One
// thread per symmetric 3 x 3 matrix: cyclic Jacobi on its symmetric part (backward stable,
// eigenvalues to a few eps ||M||, also for the repeated eigenvalues of symmetric objects),
// then the three eigenvalues in ascending order.
#include "mrom_internal.h"

#include <cfloat>

namespace mrom {
namespace {

// One Jacobi rotation annihilating a[p][q] (p < q) of the symmetric 3 x 3 matrix a.
__device__ __forceinline__ void jacobi_rotate(double (&a)[3][3], int p, int q) {
  const double apq = a[p][q];
  if (apq == 0.0) return;
  const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
  const double t = fabs(theta) > 1e150 ? 0.5 / theta
                                       : (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
  const double c = 1.0 / sqrt(fma(t, t, 1.0)), s = t * c;
  a[p][p] -= t * apq;
  a[q][q] += t * apq;
  a[p][q] = a[q][p] = 0.0;
  const int k = 3 - p - q;  // the third index
  const double akp = a[k][p], akq = a[k][q];
  a[k][p] = a[p][k] = c * akp - s * akq;
  a[k][q] = a[q][k] = s * akp + c * akq;
}

__global__ void eig3_kernel(const double* __restrict__ M, int64_t n, double* __restrict__ eig) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double* m = M + t * 9;
    double a[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) a[i][j] = 0.5 * (m[i * 3 + j] + m[j * 3 + i]);
    double fro = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) fro = fma(a[i][j], a[i][j], fro);
    for (int sweep = 0; sweep < 12; ++sweep) {
      const double off = 2.0 * (a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2]);
      if (!(off > DBL_EPSILON * DBL_EPSILON * fro)) break;  // also stops on a non-finite entry
      jacobi_rotate(a, 0, 1);
      jacobi_rotate(a, 0, 2);
      jacobi_rotate(a, 1, 2);
    }
    double e0 = a[0][0], e1 = a[1][1], e2 = a[2][2], tmp;
    if (e0 > e1) { tmp = e0; e0 = e1; e1 = tmp; }
    if (e1 > e2) { tmp = e1; e1 = e2; e2 = tmp; }
    if (e0 > e1) { tmp = e0; e0 = e1; e1 = tmp; }
    eig[t * 3 + 0] = e0;
    eig[t * 3 + 1] = e1;
    eig[t * 3 + 2] = e2;
  }
}

}  // namespace
}  // namespace mrom

using namespace mrom;

extern "C" mrom_status mrom_invariants(mrom_handle h, const double* M, int64_t n, double* eig) {
  if (!h) return MROM_EINVAL;
  if (n < 0 || (n > 0 && (!M || !eig))) return fail(h, MROM_EINVAL, "mrom_invariants: bad arguments");
  if (n == 0) return MROM_OK;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_invariants: cudaSetDevice");
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 65535LL * 8);
  eig3_kernel<<<(unsigned)blocks, 256, 0, h->stream>>>(M, n, eig);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "mrom_invariants: launch");
  ++h->launches;
  return MROM_OK;
}

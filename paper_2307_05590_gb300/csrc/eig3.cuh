// Eigenvalues of a real symmetric 3 x 3 matrix, for the rotation invariants of a spectral
// signature (Sect. 1: under a rotation Q of the object every coefficient matrix becomes Q M Q^T,
// so the eigenvalues of R~ and I are orientation independent).
//
// Smith's trigonometric solution of the characteristic cubic (O. K. Smith, "Eigenvalues of a
// symmetric 3 x 3 matrix", Comm. ACM 4 (1961) 168) gives all three eigenvalues, but near a double
// eigenvalue its arccos argument is close to +-1 and the pair loses half the digits.  The
// eigenvalue farthest from the other two (the largest when the cubic's normalised determinant is
// >= 0, else the smallest) stays accurate, so only that one is taken from the formula (its angle
// in single precision, refined by Newton's method in double precision).  Its
// eigenvector (the longest cross product of two rows of A - lambda I) deflates A onto the
// orthogonal complement, where the remaining 2 x 2 symmetric problem is solved in closed form
// (mean +- hypot).  Absolute accuracy a few eps max|a_ij|, repeated eigenvalues included.  The
// matrix is scaled by its largest entry first (no overflow or underflow in the squares).
#pragma once

#include <cmath>

namespace mrom {

__host__ __device__ inline void sym3_eig(double a11, double a22, double a33, double a12, double a13, double a23,
                                         double& e0, double& e1, double& e2) {
  const double sc = fmax(fmax(fmax(fabs(a11), fabs(a22)), fmax(fabs(a33), fabs(a12))), fmax(fabs(a13), fabs(a23)));
  if (!(sc > 0.0) || !isfinite(sc)) {  // zero matrix (or a non-finite entry: propagate it)
    e0 = e1 = e2 = sc == 0.0 ? 0.0 : a11 + a22 + a33 + a12 + a13 + a23;
    return;
  }
  const double is = 1.0 / sc;
  a11 *= is; a22 *= is; a33 *= is; a12 *= is; a13 *= is; a23 *= is;
  const double q = (a11 + a22 + a33) * (1.0 / 3.0);
  const double b11 = a11 - q, b22 = a22 - q, b33 = a33 - q;
  const double p2 = b11 * b11 + b22 * b22 + b33 * b33 + 2.0 * (a12 * a12 + a13 * a13 + a23 * a23);
  const double p = sqrt(p2 * (1.0 / 6.0));
  double lam = q;
  if (p > 0.0) {
    const double det = b11 * (b22 * b33 - a23 * a23) - a12 * (a12 * b33 - a23 * a13) + a13 * (a12 * a23 - b22 * a13);
    // r = det / (2 p^3) only feeds the single-precision angle
    const float r = fminf(1.0f, fmaxf(-1.0f, (float)det / (2.0f * (float)p * (float)p * (float)p)));
    // the angle in single precision (the FP32 units are many times the FP64 rate), then two
    // Newton steps in double precision on the depressed cubic chi(mu) = mu^3 - tr(B^2)/2 mu - det B,
    // B = A - q I, at its outermost root mu = lam - q (a simple root: chi'(mu) ~ p^2 there)
    const float phi = acosf(r) * (1.0f / 3.0f);
    const float cf = r >= 0.0f ? cosf(phi) : cosf(phi + 2.0943951f);  // + 2 pi / 3
    double mu = 2.0 * p * (double)cf;
    for (int it = 0; it < 2; ++it) {
      const double chi = fma(mu * mu - 0.5 * p2, mu, -det);
      const double dchi = fma(3.0 * mu, mu, -0.5 * p2);
      if (dchi != 0.0) mu -= chi / dchi;
    }
    lam = q + mu;
  }
  // eigenvector of lam: the longest cross product of two rows of A - lam I
  const double m00 = a11 - lam, m11 = a22 - lam, m22 = a33 - lam;
  // rows: (m00, a12, a13), (a12, m11, a23), (a13, a23, m22)
  const double c1x = a12 * a23 - a13 * m11, c1y = a13 * a12 - m00 * a23, c1z = m00 * m11 - a12 * a12;  // r0 x r1
  const double c2x = a12 * m22 - a13 * a23, c2y = a13 * a13 - m00 * m22, c2z = m00 * a23 - a12 * a13;  // r0 x r2
  const double c3x = m11 * m22 - a23 * a23, c3y = a23 * a13 - a12 * m22, c3z = a12 * a23 - m11 * a13;  // r1 x r2
  const double n1 = c1x * c1x + c1y * c1y + c1z * c1z, n2 = c2x * c2x + c2y * c2y + c2z * c2z,
               n3 = c3x * c3x + c3y * c3y + c3z * c3z;
  double vx = 1.0, vy = 0.0, vz = 0.0;
  if (n1 >= n2 && n1 >= n3 && n1 > 0.0) {
    const double in = rsqrt(n1);
    vx = c1x * in; vy = c1y * in; vz = c1z * in;
  } else if (n2 >= n3 && n2 > 0.0) {
    const double in = rsqrt(n2);
    vx = c2x * in; vy = c2y * in; vz = c2z * in;
  } else if (n3 > 0.0) {
    const double in = rsqrt(n3);
    vx = c3x * in; vy = c3y * in; vz = c3z * in;
  }
  // orthonormal u, w spanning the complement of v
  double ux, uy, uz;
  if (fabs(vx) > fabs(vy)) {
    const double in = rsqrt(fma(vx, vx, vz * vz));  // |vx| > |vy|: vx^2 + vz^2 >= 1/2
    ux = -vz * in; uy = 0.0; uz = vx * in;
  } else {
    const double in = rsqrt(fma(vy, vy, vz * vz));  // >= 1/2 as well
    ux = 0.0; uy = vz * in; uz = -vy * in;
  }
  const double wx = vy * uz - vz * uy, wy = vz * ux - vx * uz, wz = vx * uy - vy * ux;
  // the 2 x 2 matrix [u w]^T A [u w]
  const double aux = a11 * ux + a12 * uy + a13 * uz, auy = a12 * ux + a22 * uy + a23 * uz,
               auz = a13 * ux + a23 * uy + a33 * uz;
  const double awx = a11 * wx + a12 * wy + a13 * wz, awy = a12 * wx + a22 * wy + a23 * wz,
               awz = a13 * wx + a23 * wy + a33 * wz;
  const double t11 = ux * aux + uy * auy + uz * auz;
  const double t12 = ux * awx + uy * awy + uz * awz;
  const double t22 = wx * awx + wy * awy + wz * awz;
  const double hd = 0.5 * (t11 - t22);
  const double mid = 0.5 * (t11 + t22), rad = sqrt(fma(hd, hd, t12 * t12));  // entries scaled to <= 1
  double x0 = lam, x1 = mid - rad, x2 = mid + rad, tmp;
  if (x0 > x1) { tmp = x0; x0 = x1; x1 = tmp; }
  if (x1 > x2) { tmp = x1; x1 = x2; x2 = tmp; }
  if (x0 > x1) { tmp = x0; x0 = x1; x1 = tmp; }
  e0 = x0 * sc;
  e1 = x1 * sc;
  e2 = x2 * sc;
}

}  // namespace mrom

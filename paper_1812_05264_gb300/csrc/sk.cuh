// Slater-Koster two-centre blocks for an s/p/d basis (Slater & Koster, Phys. Rev. 94, 1498
// (1954), Table I), written once for a scalar type T so that the same code gives the block
// (T = double) and the block with its gradient in the bond vector (T = Dual3, forward-mode
// automatic differentiation).  Orbital order s, px, py, pz, dxy, dyz, dzx, dx2-y2, d3z2-r2;
// block(d)[i][j] couples orbital i on atom a with orbital j on atom b, d = R_b - R_a.
#pragma once
#include <math.h>

namespace tbk {

struct Dual3 {
  double v, g[3];
  __host__ __device__ Dual3() : v(0), g{0, 0, 0} {}
  __host__ __device__ Dual3(double x) : v(x), g{0, 0, 0} {}
};
__host__ __device__ inline Dual3 operator+(const Dual3& a, const Dual3& b) {
  Dual3 r; r.v = a.v + b.v;
  for (int i = 0; i < 3; ++i) r.g[i] = a.g[i] + b.g[i];
  return r;
}
__host__ __device__ inline Dual3 operator-(const Dual3& a, const Dual3& b) {
  Dual3 r; r.v = a.v - b.v;
  for (int i = 0; i < 3; ++i) r.g[i] = a.g[i] - b.g[i];
  return r;
}
__host__ __device__ inline Dual3 operator-(const Dual3& a) {
  Dual3 r; r.v = -a.v;
  for (int i = 0; i < 3; ++i) r.g[i] = -a.g[i];
  return r;
}
__host__ __device__ inline Dual3 operator*(const Dual3& a, const Dual3& b) {
  Dual3 r; r.v = a.v * b.v;
  for (int i = 0; i < 3; ++i) r.g[i] = a.g[i] * b.v + a.v * b.g[i];
  return r;
}
__host__ __device__ inline Dual3 operator*(double s, const Dual3& a) {
  Dual3 r; r.v = s * a.v;
  for (int i = 0; i < 3; ++i) r.g[i] = s * a.g[i];
  return r;
}
__host__ __device__ inline Dual3 operator/(const Dual3& a, const Dual3& b) {
  Dual3 r; r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
  for (int i = 0; i < 3; ++i) r.g[i] = (a.g[i] - r.v * b.g[i]) * ib;
  return r;
}
__host__ __device__ inline Dual3 dsqrt(const Dual3& a) {
  Dual3 r; r.v = sqrt(a.v);
  const double h = 0.5 / r.v;
  for (int i = 0; i < 3; ++i) r.g[i] = a.g[i] * h;
  return r;
}
__host__ __device__ inline Dual3 dexp(const Dual3& a) {
  Dual3 r; r.v = exp(a.v);
  for (int i = 0; i < 3; ++i) r.g[i] = a.g[i] * r.v;
  return r;
}
__host__ __device__ inline double dsqrt(double a) { return sqrt(a); }
__host__ __device__ inline double dexp(double a) { return exp(a); }

// Angular momentum of each orbital (parity of the reversed bond is (-1)^(la + lb)).
__host__ __device__ inline int sk_l(int i) { return i == 0 ? 0 : (i < 4 ? 1 : 2); }

template <class T>
__host__ __device__ inline void sk_block(const T d[3], const double V[10], double r0,
                                         double decay, T E[81]) {
  const double s3 = 1.7320508075688772;  // sqrt(3)
  const T r = dsqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const T l = d[0] / r, m = d[1] / r, n = d[2] / r;
  const T f = dexp(-decay * (r / T(r0) - T(1.0)));
  T v[10];
  for (int i = 0; i < 10; ++i) v[i] = V[i] * f;
  const T &sss = v[0], &sps = v[1], &sds = v[2], &pps = v[3], &ppp = v[4], &pds = v[5],
          &pdp = v[6], &dds = v[7], &ddp = v[8], &ddd = v[9];
  const T ll = l * l, mm = m * m, nn = n * n, one(1.0);
  const T lm = l * m, mn = m * n, nl = n * l, lmn = lm * n;
  const T amb = ll - mm;                 // l^2 - m^2
  const T z2 = nn - 0.5 * (ll + mm);     // n^2 - (l^2 + m^2)/2
  const T dir[3] = {l, m, n};
  const T sq[3] = {ll, mm, nn};
  // s row
  E[0] = sss;
  for (int a = 0; a < 3; ++a) E[1 + a] = dir[a] * sps;
  E[4] = s3 * lm * sds;
  E[5] = s3 * mn * sds;
  E[6] = s3 * nl * sds;
  E[7] = (0.5 * s3) * amb * sds;
  E[8] = z2 * sds;
  // p-p: d_a d_b (pps - ppp) + delta_ab ppp
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) {
      T e = dir[a] * dir[b] * (pps - ppp);
      if (a == b) e = e + ppp;
      E[9 * (1 + a) + 1 + b] = e;
    }
  // p-d.  For p_a against d_xy-like orbitals (pairs (x,y)=4, (y,z)=5, (z,x)=6):
  //   p_a . d_bc = sqrt3 d_a d_b d_c pds + (delta_ab d_c + delta_ac d_b - 2 d_a d_b d_c) pdp
  const int pr[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  for (int a = 0; a < 3; ++a)
    for (int q = 0; q < 3; ++q) {
      const int b = pr[q][0], c = pr[q][1];
      const T abc = dir[a] * dir[b] * dir[c];
      T e = s3 * abc * pds - 2.0 * abc * pdp;
      if (a == b) e = e + dir[c] * pdp;
      if (a == c) e = e + dir[b] * pdp;
      E[9 * (1 + a) + 4 + q] = e;
    }
  // p - d(x2-y2)
  E[9 * 1 + 7] = (0.5 * s3) * l * amb * pds + l * (one - amb) * pdp;
  E[9 * 2 + 7] = (0.5 * s3) * m * amb * pds - m * (one + amb) * pdp;
  E[9 * 3 + 7] = (0.5 * s3) * n * amb * pds - n * amb * pdp;
  // p - d(3z2-r2)
  E[9 * 1 + 8] = l * z2 * pds - s3 * l * nn * pdp;
  E[9 * 2 + 8] = m * z2 * pds - s3 * m * nn * pdp;
  E[9 * 3 + 8] = n * z2 * pds + s3 * n * (ll + mm) * pdp;
  // d_xy-like with d_xy-like (diagonal): 3 a^2 b^2 dds + (a^2 + b^2 - 4 a^2 b^2) ddp +
  // (c^2 + a^2 b^2) ddd, with (a, b, c) = (l, m, n), (m, n, l), (n, l, m)
  for (int q = 0; q < 3; ++q) {
    const int a = pr[q][0], b = pr[q][1], c = 3 - a - b;
    const T a2b2 = sq[a] * sq[b];
    E[9 * (4 + q) + 4 + q] = 3.0 * a2b2 * dds + (sq[a] + sq[b] - 4.0 * a2b2) * ddp + (sq[c] + a2b2) * ddd;
  }
  // off-diagonal d_xy-like pairs: (xy,yz), (xy,zx), (yz,zx).  For orbitals sharing the
  // coordinate k, with the other two coordinates i (first) and j (second):
  //   3 i k^2 j dds + i j (1 - 4 k^2) ddp + i j (k^2 - 1) ddd
  {
    // (xy, yz): shared y, others x, z
    E[9 * 4 + 5] = 3.0 * l * mm * n * dds + nl * (one - 4.0 * mm) * ddp + nl * (mm - one) * ddd;
    // (xy, zx): shared x, others y, z
    E[9 * 4 + 6] = 3.0 * ll * mn * dds + mn * (one - 4.0 * ll) * ddp + mn * (ll - one) * ddd;
    // (yz, zx): shared z, others y, x
    E[9 * 5 + 6] = 3.0 * lm * nn * dds + lm * (one - 4.0 * nn) * ddp + lm * (nn - one) * ddd;
  }
  // d_xy-like with d(x2-y2)
  E[9 * 4 + 7] = 1.5 * lm * amb * dds - 2.0 * lm * amb * ddp + 0.5 * lm * amb * ddd;
  E[9 * 5 + 7] = 1.5 * mn * amb * dds - mn * (one + 2.0 * amb) * ddp + mn * (one + 0.5 * amb) * ddd;
  E[9 * 6 + 7] = 1.5 * nl * amb * dds + nl * (one - 2.0 * amb) * ddp - nl * (one - 0.5 * amb) * ddd;
  // d_xy-like with d(3z2-r2)
  E[9 * 4 + 8] = s3 * lm * z2 * dds - 2.0 * s3 * lm * nn * ddp + (0.5 * s3) * lm * (one + nn) * ddd;
  E[9 * 5 + 8] = s3 * mn * z2 * dds + s3 * mn * (ll + mm - nn) * ddp - (0.5 * s3) * mn * (ll + mm) * ddd;
  E[9 * 6 + 8] = s3 * nl * z2 * dds + s3 * nl * (ll + mm - nn) * ddp - (0.5 * s3) * nl * (ll + mm) * ddd;
  // e_g block
  E[9 * 7 + 7] = 0.75 * amb * amb * dds + (ll + mm - amb * amb) * ddp + (nn + 0.25 * amb * amb) * ddd;
  E[9 * 7 + 8] = (0.5 * s3) * amb * z2 * dds - s3 * nn * amb * ddp + (0.25 * s3) * (one + nn) * amb * ddd;
  E[9 * 8 + 8] = z2 * z2 * dds + 3.0 * nn * (ll + mm) * ddp + 0.75 * (ll + mm) * (ll + mm) * ddd;
  // lower triangle from the parity of the reversed bond
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < i; ++j) {
      const T u = E[9 * j + i];
      E[9 * i + j] = ((sk_l(i) + sk_l(j)) & 1) ? -u : u;
    }
}

}  // namespace tbk

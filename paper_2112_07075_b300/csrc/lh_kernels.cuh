// Templated CUDA kernels of liblh for one (DIM, P, Q) = (dimension, H1 order,
// Gauss points per direction) combination. Every kernel is element-batched:
// a CTA owns NB consecutive elements, stages their DOFs and quadrature data in
// shared memory and applies the 1D basis tables one axis at a time (sum
// factorization, arXiv 2112.07075 Section 3.2). Element results that belong to
// shared H1 nodes go to an element vector (E-vector) and are summed per node by
// a deterministic gather (the G^T of Section 3.1), so results are bit-identical
// from run to run.
#pragma once

#include "lh_device.cuh"
#include "lh_internal.h"

namespace lh {

// ---------------------------------------------------------------------------
// Structured-mesh index maps (layouts documented in include/lh.h).
// ---------------------------------------------------------------------------
template <int DIM, int D>
__device__ __forceinline__ int h1_node(const MeshDesc &m, int e, int i) {
  constexpr int P = D - 1;
  const int ex = e % m.nx;
  const int t = e / m.nx;
  const int ix = i % D;
  if constexpr (DIM == 2) {
    const int ey = t;
    const int iy = i / D;
    return (ex * P + ix) + m.n1x * (ey * P + iy);
  } else {
    const int ey = t % m.ny, ez = t / m.ny;
    const int iy = (i / D) % D, iz = i / (D * D);
    return (ex * P + ix) + m.n1x * ((ey * P + iy) + m.n1y * (ez * P + iz));
  }
}

// Contributions of element-local nodes to H1 node coordinate gc along one axis.
__device__ __forceinline__ int axis_owners(int gc, int P, int nel, int (&ee)[2], int (&ii)[2]) {
  const int e = gc / P, i = gc - e * P;
  if (i != 0) {
    ee[0] = e;
    ii[0] = i;
    return 1;
  }
  int n = 0;
  if (e > 0) { ee[n] = e - 1; ii[n] = P; ++n; }
  if (e < nel) { ee[n] = e; ii[n] = 0; ++n; }
  return n;
}

// Global H1 node of element e's local node (0,0,0): the element's base node.
template <int DIM, int D>
__device__ __forceinline__ int h1_base(const MeshDesc &m, int e) {
  constexpr int P = D - 1;
  const int ex = e % m.nx, t = e / m.nx;
  if constexpr (DIM == 2) return ex * P + m.n1x * (t * P);
  else return ex * P + m.n1x * ((t % m.ny) * P + m.n1y * ((t / m.ny) * P));
}
// Offset of local node i from the element's base node (compile-time divisions only).
template <int DIM, int D>
__device__ __forceinline__ int h1_local(const MeshDesc &m, int i) {
  if constexpr (DIM == 2) return i % D + m.n1x * (i / D);
  else return i % D + m.n1x * ((i / D) % D + m.n1y * (i / (D * D)));
}

// Offsets e*C*ND + i of every element-local copy of node g in an E-vector with C
// components (add c*ND for component c), in a fixed order; returns their count.
template <int DIM, int D>
__device__ __forceinline__ int node_copies(const MeshDesc &m, int g, int C, int (&off)[1 << DIM]) {
  constexpr int P = D - 1, ND = ipow<D, DIM>::value;
  int ex[2], ix[2], ey[2], iy[2], ez[2] = {0, 0}, iz[2] = {0, 0};
  const int gx = g % m.n1x;
  const int t = g / m.n1x;
  const int nxo = axis_owners(gx, P, m.nx, ex, ix);
  int nyo, nzo = 1;
  if constexpr (DIM == 2) {
    nyo = axis_owners(t, P, m.ny, ey, iy);
  } else {
    nyo = axis_owners(t % m.n1y, P, m.ny, ey, iy);
    nzo = axis_owners(t / m.n1y, P, m.nz, ez, iz);
  }
  int n = 0;
  for (int a = 0; a < nzo; ++a)
    for (int b = 0; b < nyo; ++b)
      for (int k = 0; k < nxo; ++k) {
        const int e = ex[k] + m.nx * (ey[b] + m.ny * ez[a]);
        const int i = ix[k] + D * (iy[b] + D * iz[a]);
        off[n++] = e * C * ND + i;
      }
  return n;
}

// Offsets e*C*ND + i of node g's element copies, computed from the node's grid
// coordinates (no table read): position j = (a*2 + b)*2 + k picks the z, y, x
// owner (2D: j = b*2 + k); -1 where that axis has a single owner. Position 0 is
// always a copy, and the valid positions come in the order of node_copies (and of
// the node-copy table), so sums over the copies in position order are the same.
template <int DIM, int D>
__device__ __forceinline__ void node_offsets(const MeshDesc &m, int g, int C, int (&off)[1 << DIM]) {
  constexpr int P = D - 1, ND = ipow<D, DIM>::value;
  // along one axis: the first owner (element e-1 at local index P when the node
  // sits on an element boundary other than the first, else element e at index i)
  // and the second (element e at index 0) if the boundary is interior
  auto axis = [](int gc, int nel, int se, int si, int &o0, int &o1) {
    const int e = gc / P, i = gc - e * P;
    const bool lo = i == 0 && e > 0;
    o0 = (lo ? e - 1 : e) * se + (lo ? P : i) * si;
    o1 = lo && e < nel ? e * se : -1;
  };
  const int gx = g % m.n1x, t = g / m.n1x;
  int x0, x1, y0, y1;
  axis(gx, m.nx, C * ND, 1, x0, x1);
  if constexpr (DIM == 2) {
    axis(t, m.ny, m.nx * C * ND, D, y0, y1);
    off[0] = x0 + y0;
    off[1] = x1 >= 0 ? x1 + y0 : -1;
    off[2] = y1 >= 0 ? x0 + y1 : -1;
    off[3] = x1 >= 0 && y1 >= 0 ? x1 + y1 : -1;
  } else {
    int z0, z1;
    axis(t % m.n1y, m.ny, m.nx * C * ND, D, y0, y1);
    axis(t / m.n1y, m.nz, m.nx * m.ny * C * ND, D * D, z0, z1);
    const int xs[2] = {x0, x1}, ys[2] = {y0, y1}, zs[2] = {z0, z1};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int k = 0; k < 2; ++k)
          off[(a * 2 + b) * 2 + k] = xs[k] >= 0 && ys[b] >= 0 && zs[a] >= 0 ? xs[k] + ys[b] + zs[a] : -1;
  }
}

// Row g of the node-copy table (offsets e*DIM*ND + i of node g's copies, -1 padded).
template <int DIM>
__device__ __forceinline__ void node_table_row(const int *__restrict__ tab, int g, int (&off)[1 << DIM]) {
  const int4 a = __ldg(reinterpret_cast<const int4 *>(tab + (size_t)g * (1 << DIM)));
  off[0] = a.x; off[1] = a.y; off[2] = a.z; off[3] = a.w;
  if constexpr (DIM == 3) {
    const int4 b = __ldg(reinterpret_cast<const int4 *>(tab + (size_t)g * 8 + 4));
    off[4] = b.x; off[5] = b.y; off[6] = b.z; off[7] = b.w;
  }
}

// Is H1 node g constrained for velocity component c (v.n = 0 on the box faces)?
template <int DIM>
__device__ __forceinline__ bool h1_constrained(const MeshDesc &m, int g, int c) {
  const int gx = g % m.n1x;
  if (c == 0) return gx == 0 || gx == m.n1x - 1;
  const int t = g / m.n1x;
  if constexpr (DIM == 2) {
    return t == 0 || t == m.n1y - 1;
  } else {
    if (c == 1) {
      const int gy = t % m.n1y;
      return gy == 0 || gy == m.n1y - 1;
    }
    const int gz = t / m.n1y;
    return gz == 0 || gz == m.n1z - 1;
  }
}

// Sum over the elements sharing node g of evec[e][c][i] (fixed order). evec is
// deliberately not __restrict__: inside the persistent CG kernel other blocks
// write it between grid barriers, so it must not be read through the
// non-coherent read-only path.
template <int DIM, int D, typename T = double>
__device__ __forceinline__ T gather_node(const MeshDesc &m, const T *evec, int C, int c, int g) {
  constexpr int P = D - 1, ND = ipow<D, DIM>::value;
  int ex[2], ix[2], ey[2], iy[2], ez[2] = {0, 0}, iz[2] = {0, 0};
  const int gx = g % m.n1x;
  const int t = g / m.n1x;
  const int nxo = axis_owners(gx, P, m.nx, ex, ix);
  int nyo, nzo = 1;
  if constexpr (DIM == 2) {
    nyo = axis_owners(t, P, m.ny, ey, iy);
  } else {
    nyo = axis_owners(t % m.n1y, P, m.ny, ey, iy);
    nzo = axis_owners(t / m.n1y, P, m.nz, ez, iz);
  }
  T s = 0;
  for (int a = 0; a < nzo; ++a)
    for (int b = 0; b < nyo; ++b)
      for (int k = 0; k < nxo; ++k) {
        const int e = ex[k] + m.nx * (ey[b] + m.ny * ez[a]);
        const int i = ix[k] + D * (iy[b] + D * iz[a]);
        s += evec[((size_t)e * C + c) * ND + i];
      }
  return s;
}

// ---------------------------------------------------------------------------
// Per-qpoint physics (reading of Sections 2.1 and 6):
// EOS, tensor artificial viscosity, stress, force data and time-step bound.
// ---------------------------------------------------------------------------
constexpr double kEps0 = 1.0e-12;
constexpr double kDegen = 1.0e-14;

__device__ __forceinline__ double smooth_step01(double x, double e0) {
  double y = (x + e0) / (2.0 * e0);
  y = fmin(fmax(y, 0.0), 1.0);
  return y * y * (3.0 - 2.0 * y);
}

// Smallest eigenvalue of a symmetric 2x2 (a b; b c) and, if s != nullptr, its unit eigenvector.
__device__ __forceinline__ double eig_min2(double a, double b, double c, double *s) {
  const double hd = 0.5 * (a - c);
  const double lam = 0.5 * (a + c) - sqrt(hd * hd + b * b);
  if (s) {
    const double r0x = a - lam, r0y = b, r1x = b, r1y = c - lam;
    const double n0 = sqrt(r0x * r0x + r0y * r0y), n1 = sqrt(r1x * r1x + r1y * r1y);
    const bool first = n0 >= n1;
    const double rx = first ? r0x : r1x, ry = first ? r0y : r1y, nr = first ? n0 : n1;
    const double nA = sqrt(a * a + 2.0 * b * b + c * c);
    if (nr <= kDegen * nA) {
      s[0] = 1.0;
      s[1] = 0.0;
    } else {
      s[0] = -ry / nr;
      s[1] = rx / nr;
    }
  }
  return lam;
}

// Smallest root mu of the characteristic polynomial of the trace-free symmetric
// B = A - qI (diagonal d0, d1, d2; off-diagonal a01, a02, a12; p2 = tr B^2):
// f(mu) = det(B - mu I) = -mu^3 + (p2 / 2) mu + det B. B is first scaled by a power
// of two s with s^2 p2 in [1, 4) (exact), so the FP32 parts below neither underflow
// nor overflow whatever the magnitude of A. Seed: the trigonometric closed form
// evaluated in FP32 (cheap on B300, where FP64 runs at 1/64 of the FP32 rate);
// then two Newton steps t -= f(t) / f'(t) in FP64 on the scaled polynomial (Newton's
// method for a simple polynomial root; the step uses an FP32 reciprocal of f', which
// changes only the quadratic convergence constant: each step still squares the
// relative error down to rounding). Returns false when the root is not well
// separated, |f'(t0)| < 0.05 tr (sB)^2 (a double or triple smallest eigenvalue), or
// p2 is zero, subnormal or not finite: f is then flat near the root (or there is
// nothing to refine) and the caller takes the FP64 trigonometric form. Where it
// returns true the root is accurate to a few units of rounding of sqrt(p2).
__device__ __forceinline__ bool eig_min3_newton(double d0, double d1, double d2, double a01, double a02, double a12,
                                                double p2, double &mu) {
  if (!(p2 > 1e-300) || !(p2 < 1e300)) return false;
  const int ex = ((__double2hiint(p2) >> 20) & 0x7ff) - 1023;   // p2 = m 2^ex, m in [1, 2)
  const int h = ex >> 1;                                        // floor(ex / 2)
  const double sc = __hiloint2double((1023 - h) << 20, 0);      // 2^-h
  const double e0 = d0 * sc, e1 = d1 * sc, e2 = d2 * sc, e01 = a01 * sc, e02 = a02 * sc, e12 = a12 * sc;
  const double q2 = p2 * sc * sc;                               // tr (sB)^2 in [1, 4)
  const float ppf = sqrtf((float)q2 * (1.0f / 6.0f)), ipf = 1.0f / ppf;
  const float b00 = (float)e0 * ipf, b11 = (float)e1 * ipf, b22 = (float)e2 * ipf;
  const float b01 = (float)e01 * ipf, b02 = (float)e02 * ipf, b12 = (float)e12 * ipf;
  const float detbf = b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
  const float rf = fminf(fmaxf(0.5f * detbf, -1.0f), 1.0f);
  double t = (double)(2.0f * ppf * __cosf(acosf(rf) * (1.0f / 3.0f) + 2.0943951f));
  const double c1 = 0.5 * q2;
  double fp = fma(-3.0 * t, t, c1);
  if (!(fabs(fp) >= 0.05 * q2)) return false;
  const double detB = e0 * (e1 * e2 - e12 * e12) - e01 * (e01 * e2 - e12 * e02) + e02 * (e01 * e12 - e1 * e02);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double f = fma(fma(-t, t, c1), t, detB);
    fp = fma(-3.0 * t, t, c1);
    t = fma(-f, (double)(1.0f / (float)fp), t);
  }
  mu = t * __hiloint2double((1023 + h) << 20, 0);               // t / s
  return true;
}

// Smallest eigenvalue of a symmetric 3x3 (A[0..8], row-major, symmetric) and, if
// s != nullptr, its unit eigenvector from the largest cross product of two rows of
// (A - lam I). The eigenvalue: Newton-polished root of the characteristic cubic
// (eig_min3_newton) where it is well separated, else the FP64 trigonometric closed
// form (Smith 1961).
__device__ __forceinline__ double eig_min3(const double *A, double *s) {
  const double a00 = A[0], a01 = A[1], a02 = A[2], a11 = A[4], a12 = A[5], a22 = A[8];
  constexpr double third = 1.0 / 3.0, sixth = 1.0 / 6.0;
  const double q = (a00 + a11 + a22) * third;
  const double p1 = a01 * a01 + a02 * a02 + a12 * a12;
  const double d0 = a00 - q, d1 = a11 - q, d2 = a22 - q;
  const double p2 = d0 * d0 + d1 * d1 + d2 * d2 + 2.0 * p1;
  double lam = q, mu;
  if (eig_min3_newton(d0, d1, d2, a01, a02, a12, p2, mu)) {
    lam = q + mu;
  } else {
    const double pp = sqrt(p2 * sixth);
    if (pp > 0.0) {
      const double ip = 1.0 / pp;
      const double b00 = d0 * ip, b11 = d1 * ip, b22 = d2 * ip, b01 = a01 * ip, b02 = a02 * ip, b12 = a12 * ip;
      const double detb =
          b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02);
      const double r = fmin(fmax(0.5 * detb, -1.0), 1.0);
      const double phi = acos(r) * third;
      lam = q + 2.0 * pp * cos(phi + 2.0943951023931957);  // 2*pi/3
    }
  }
  if (s) {
    const double m00 = a00 - lam, m11 = a11 - lam, m22 = a22 - lam;
    const double r0[3] = {m00, a01, a02}, r1[3] = {a01, m11, a12}, r2[3] = {a02, a12, m22};
    double cr[3][3];
    const double *ra[3] = {r0, r0, r1}, *rb[3] = {r1, r2, r2};
    double nbest = -1.0;
    int kbest = 0;
    // candidates compared by squared norm; one square root for the chosen one
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      cr[k][0] = ra[k][1] * rb[k][2] - ra[k][2] * rb[k][1];
      cr[k][1] = ra[k][2] * rb[k][0] - ra[k][0] * rb[k][2];
      cr[k][2] = ra[k][0] * rb[k][1] - ra[k][1] * rb[k][0];
      const double n2 = cr[k][0] * cr[k][0] + cr[k][1] * cr[k][1] + cr[k][2] * cr[k][2];
      if (n2 > nbest) { nbest = n2; kbest = k; }
    }
    const double nM2 = m00 * m00 + m11 * m11 + m22 * m22 + 2.0 * (a01 * a01 + a02 * a02 + a12 * a12);
    const double dthr = kDegen * nM2;
    if (nbest <= dthr * dthr) {
      const double nM = sqrt(nM2);
      const double nA = sqrt(a00 * a00 + a11 * a11 + a22 * a22 + 2.0 * p1);
      if (nM <= kDegen * nA || nM == 0.0) {
        s[0] = 1.0; s[1] = 0.0; s[2] = 0.0;
      } else {
        const double *rows[3] = {r0, r1, r2};
        int rb_i = 0;
        double rn = -1.0;
        for (int k = 0; k < 3; ++k) {
          const double n = sqrt(rows[k][0] * rows[k][0] + rows[k][1] * rows[k][1] + rows[k][2] * rows[k][2]);
          if (n > rn) { rn = n; rb_i = k; }
        }
        const double *rv = rows[rb_i];
        int kk = 0;
        double amin = fabs(rv[0]);
        if (fabs(rv[1]) < amin) { amin = fabs(rv[1]); kk = 1; }
        if (fabs(rv[2]) < amin) { kk = 2; }
        // rv x e_kk
        double c0, c1, c2;
        if (kk == 0) { c0 = 0.0; c1 = rv[2]; c2 = -rv[1]; }
        else if (kk == 1) { c0 = -rv[2]; c1 = 0.0; c2 = rv[0]; }
        else { c0 = rv[1]; c1 = -rv[0]; c2 = 0.0; }
        const double n = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
        s[0] = c0 / n; s[1] = c1 / n; s[2] = c2 / n;
      }
    } else {
      const double inv = 1.0 / sqrt(nbest);
      s[0] = cr[kbest][0] * inv;
      s[1] = cr[kbest][1] * inv;
      s[2] = cr[kbest][2] * inv;
    }
  }
  return lam;
}

struct QPointOut {
  double inv_dt;   // 1/dt_q (before the CFL factor); +inf if inverted
  bool inverted;
};

// J, Ji0, dV: row-major DIM x DIM. J[c][l] = dx_c/dxi_l, dV[c][l] = dv_c/dxi_l.
// m = omega * rho0 * detJ0, w = omega, iw = 1/omega. Writes D[c*DIM+l].
template <int DIM>
__device__ __forceinline__ QPointOut qpoint_physics(const double *J, const double *Ji0, const double *dV, double e_q,
                                                    double m, double w, double iw, const PhysParams &pp,
                                                    bool want_dt, double *Dout) {
  QPointOut o;
  double Ji[DIM * DIM];
  double det, id;
  if constexpr (DIM == 2) {
    det = J[0] * J[3] - J[1] * J[2];
    id = 1.0 / det;
    Ji[0] = J[3] * id; Ji[1] = -J[1] * id; Ji[2] = -J[2] * id; Ji[3] = J[0] * id;
  } else {
    const double c00 = J[4] * J[8] - J[5] * J[7];
    const double c01 = J[5] * J[6] - J[3] * J[8];
    const double c02 = J[3] * J[7] - J[4] * J[6];
    det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    id = 1.0 / det;
    Ji[0] = c00 * id; Ji[1] = (J[2] * J[7] - J[1] * J[8]) * id; Ji[2] = (J[1] * J[5] - J[2] * J[4]) * id;
    Ji[3] = c01 * id; Ji[4] = (J[0] * J[8] - J[2] * J[6]) * id; Ji[5] = (J[2] * J[3] - J[0] * J[5]) * id;
    Ji[6] = c02 * id; Ji[7] = (J[1] * J[6] - J[0] * J[7]) * id; Ji[8] = (J[0] * J[4] - J[1] * J[3]) * id;
  }
  o.inverted = !(det > 0.0);
  const double rho = m * iw * id;
  const double ep = fmax(e_q, 0.0);
  const double pres = (pp.gamma - 1.0) * rho * ep;
  const double cs = sqrt(pp.gamma * (pp.gamma - 1.0) * ep);
  // grad v = dV Jinv, strain = sym part
  double gv[DIM * DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      double s = dV[c * DIM] * Ji[b];
#pragma unroll
      for (int l = 1; l < DIM; ++l) s = fma(dV[c * DIM + l], Ji[l * DIM + b], s);
      gv[c * DIM + b] = s;
    }
  double eps[DIM * DIM];   // symmetric: the upper triangle is computed and mirrored
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int b = c; b < DIM; ++b) {
      const double v = 0.5 * (gv[c * DIM + b] + gv[b * DIM + c]);
      eps[c * DIM + b] = v;
      eps[b * DIM + c] = v;
    }
  double sigma[DIM * DIM];
#pragma unroll
  for (int k = 0; k < DIM * DIM; ++k) sigma[k] = 0.0;
#pragma unroll
  for (int c = 0; c < DIM; ++c) sigma[c * DIM + c] = -pres;
  double mu = 0.0;
  if (pp.use_viscosity) {
    double s[DIM];
    double lam;
    if constexpr (DIM == 2) lam = eig_min2(eps[0], eps[1], eps[3], s);
    else lam = eig_min3(eps, s);
    // h = h0 |J Ji0 s|
    double t[DIM], hv[DIM];
#pragma unroll
    for (int l = 0; l < DIM; ++l) {
      double a = Ji0[l * DIM] * s[0];
#pragma unroll
      for (int b = 1; b < DIM; ++b) a = fma(Ji0[l * DIM + b], s[b], a);
      t[l] = a;
    }
    double hn2 = 0.0;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double a = J[c * DIM] * t[0];
#pragma unroll
      for (int l = 1; l < DIM; ++l) a = fma(J[c * DIM + l], t[l], a);
      hv[c] = a;
      hn2 = fma(a, a, hn2);
    }
    const double h = pp.h0 * sqrt(hn2);
    mu = 2.0 * rho * h * h * fabs(lam) + 0.5 * rho * h * cs * (1.0 - smooth_step01(lam - 2.0 * kEps0, kEps0));
#pragma unroll
    for (int k = 0; k < DIM * DIM; ++k) sigma[k] = fma(mu, eps[k], sigma[k]);
  }
  // D = w detJ sigma Jinv^T
  const double wd = w * det;
#pragma unroll
  for (int c = 0; c < DIM; ++c)
#pragma unroll
    for (int l = 0; l < DIM; ++l) {
      double a = sigma[c * DIM] * Ji[l * DIM];
#pragma unroll
      for (int b = 1; b < DIM; ++b) a = fma(sigma[c * DIM + b], Ji[l * DIM + b], a);
      Dout[c * DIM + l] = wd * a;
    }
  o.inv_dt = 0.0;
  if (want_dt) {
    double lamJ;
    if constexpr (DIM == 2) {
      const double a = J[0] * J[0] + J[2] * J[2], b = J[0] * J[1] + J[2] * J[3], c = J[1] * J[1] + J[3] * J[3];
      lamJ = eig_min2(a, b, c, nullptr);
    } else {
      double JtJ[9];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int b = c; b < 3; ++b) {
          const double v = J[c] * J[b] + J[3 + c] * J[3 + b] + J[6 + c] * J[6 + b];
          JtJ[c * 3 + b] = v;
          JtJ[b * 3 + c] = v;
        }
      lamJ = eig_min3(JtJ, nullptr);
    }
    // h_min = sqrt(lamJ) / p; 1/dt = c_s / h_min + 2.5 mu / (rho h_min^2), one division
    const double l2 = fmax(lamJ, 0.0);
    const double hm = sqrt(l2);   // p h_min
    o.inv_dt = pp.order * (cs * rho * hm + 2.5 * pp.order * mu) / (rho * l2);
    if (o.inverted) o.inv_dt = INFINITY;
  }
  return o;
}

// ---------------------------------------------------------------------------
// The kernel family for one (DIM, P, Q).
// ---------------------------------------------------------------------------
template <int DIM, int P, int Q>
struct Family {
  static constexpr int D = P + 1;
  static constexpr int L = P;
  static constexpr int ND = ipow<D, DIM>::value;
  static constexpr int NL = ipow<L, DIM>::value;
  static constexpr int NQ = ipow<Q, DIM>::value;
  static constexpr int NB = NQ >= 128 ? 1 : (256 / NQ);   // elements per CTA
  static constexpr int THREADS = ((NB * NQ < 256 ? NB * NQ : 256) + 31) / 32 * 32;
  // basis table layout (doubles): B[Q][D] G[Q][D] Bt[D][Q] Gt[D][Q] Bl[Q][L] Blt[L][Q]
  // B2t[D][Q] (squared B, transposed) w[Q] 1/w[Q] gll[D]
  static constexpr int oB = 0, oG = Q * D, oBt = 2 * Q * D, oGt = 3 * Q * D, oBl = 4 * Q * D,
                       oBlt = 4 * Q * D + Q * L, oB2t = 4 * Q * D + 2 * Q * L, oW = 5 * Q * D + 2 * Q * L,
                       oIW = oW + Q, oZ = oIW + Q;
  static constexpr int TAB = ((oZ + D) + 1) / 2 * 2;
  static constexpr int RED_NV = 8;          // block_sum<NV> needs 32*NV doubles: NV <= RED_NV
  static constexpr int RED = RED_NV * 32;   // reduction scratch (doubles)

  static constexpr int CX = NB * DIM;        // one H1 vector field of NB elements
  static constexpr int C2X = NB * 2 * DIM;   // two H1 vector fields
  static constexpr int max3(int a, int b, int c) { return a > b ? (a > c ? a : c) : (b > c ? b : c); }

  template <int NV>
  static __device__ __forceinline__ void bsum(double (&v)[NV], double *red) {
    static_assert(NV <= RED_NV, "reduction scratch too small");
    block_sum<NV>(v, red);
  }

  static __device__ __forceinline__ void load_tab(double *s, const double *__restrict__ tab) {
    for (int k = threadIdx.x; k < oZ + D; k += blockDim.x) s[k] = tab[k];
  }
  static __device__ __forceinline__ void qweight(const double *st, int q, double &w, double &iw) {
    const int qx = q % Q;
    if constexpr (DIM == 2) {
      const int qy = q / Q;
      w = st[oW + qx] * st[oW + qy];
      iw = st[oIW + qx] * st[oIW + qy];
    } else {
      const int qy = (q / Q) % Q, qz = q / (Q * Q);
      w = st[oW + qx] * st[oW + qy] * st[oW + qz];
      iw = st[oIW + qx] * st[oIW + qy] * st[oIW + qz];
    }
  }
  // gather C_ = NB*ncomp components of an H1 vector field into u[b*ncomp + c][i]
  static __device__ __forceinline__ void gather_elem(double *u, const double *__restrict__ f, int ncomp,
                                                     const MeshDesc &m, int e0, int nb) {
    for (int k = threadIdx.x; k < NB * ncomp * ND; k += blockDim.x) {
      const int i = k % ND, bc = k / ND, c = bc % ncomp, b = bc / ncomp;
      u[k] = b < nb ? f[(size_t)c * m.nh1 + h1_node<DIM, D>(m, e0 + b, i)] : 0.0;
    }
  }
  static __device__ __forceinline__ void apply_me_inv(const double *__restrict__ me_inv, const double *rhs, int e,
                                                      int j, double &s) {
    const double *Mi = me_inv + ((size_t)e * NL + j) * NL;
    s = Mi[0] * rhs[0];
    for (int kk = 1; kk < NL; ++kk) s = fma(Mi[kk], rhs[kk], s);
  }

  // ===== quadrature data (rows a1-a7) =====================================
  // smem: tab | u[C2X][ND] | S (grad scratch C2X) | g[DIM][C2X][NQ] | eq[NB][NQ] | el[NB][NL] | red
  static constexpr int QD_S = max3(grad_scratch<DIM, D, Q>(C2X), interp_scratch<DIM, L, Q>(NB), 0);
  static constexpr size_t qdata_smem() {
    return sizeof(double) * (TAB + C2X * ND + QD_S + DIM * C2X * NQ + NB * NQ + NB * NL + RED);
  }
  static __device__ __forceinline__ void body_qdata(const QdataArgs &a, int e0) {
    extern __shared__ double sm[];
    double *st = sm, *u = st + TAB, *S = u + C2X * ND, *g = S + QD_S, *eq = g + DIM * C2X * NQ;
    double *el = eq + NB * NQ, *red = el + NB * NL;
    const MeshDesc &m = a.mesh;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    for (int k = threadIdx.x; k < C2X * ND; k += blockDim.x) {
      const int i = k % ND, bc = k / ND, c = bc % (2 * DIM), b = bc / (2 * DIM);
      double val = 0.0;
      if (b < nb) {
        const int gi = h1_node<DIM, D>(m, e0 + b, i);
        val = c < DIM ? a.x[(size_t)c * m.nh1 + gi] : a.v[(size_t)(c - DIM) * m.nh1 + gi];
      }
      u[k] = val;
    }
    for (int k = threadIdx.x; k < NB * NL; k += blockDim.x)
      el[k] = k / NL < nb ? a.e[(size_t)e0 * NL + k] : 0.0;
    __syncthreads();
    interp<DIM, L, Q, NB>(el, eq, S, st + oBl);   // energy at qpoints
    grad_ref<DIM, D, Q, C2X>(u, g, S, st + oB, st + oG);
    double inv_dt_max = 0.0;
    for (int k = threadIdx.x; k < nb * NQ; k += blockDim.x) {
      const int b = k / NQ, q = k % NQ;
      const size_t e = (size_t)(e0 + b);
      double J[DIM * DIM], dV[DIM * DIM], Ji0[DIM * DIM], Dq[DIM * DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int l = 0; l < DIM; ++l) {
          J[c * DIM + l] = g[(l * C2X + b * 2 * DIM + c) * NQ + q];
          dV[c * DIM + l] = g[(l * C2X + b * 2 * DIM + DIM + c) * NQ + q];
        }
#pragma unroll
      for (int r = 0; r < DIM * DIM; ++r) Ji0[r] = a.jinv0[(e * DIM * DIM + r) * NQ + q];
      double w, iw;
      qweight(st, q, w, iw);
      const QPointOut o = qpoint_physics<DIM>(J, Ji0, dV, eq[k], a.mq[e * NQ + q], w, iw, a.phys, a.want_dt, Dq);
      if (o.inverted) latch_status(a.status, 4);
#pragma unroll
      for (int r = 0; r < DIM * DIM; ++r) a.D[(e * DIM * DIM + r) * NQ + q] = Dq[r];
      inv_dt_max = fmax(inv_dt_max, o.inv_dt);
    }
    if (!a.want_dt) return;
    // grid max of 1/dt: per-block partial; the last block to finish reduces (fixed order).
    const double bm = block_max(inv_dt_max, red);
    __shared__ int s_last;
    if (threadIdx.x == 0) {
      a.partials[blockIdx.x] = bm;
      __threadfence();
      s_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x >= 32) return;
    __threadfence();
    double mx = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) mx = fmax(mx, ((volatile double *)a.partials)[i]);
    mx = warp_max(mx);
    if (threadIdx.x == 0) {
      *a.counter = 0u;
      const double dt_est = mx > 0.0 ? a.cfl / mx : (mx == 0.0 ? INFINITY : 0.0);
      if (a.dt_est_out) *a.dt_est_out = dt_est;
      if (a.step) {
        lh_step_info *s = a.step;
        if (a.ctl == 2) {   // half-step state: accept or reject the attempt
          const double dt = s->dt;
          s->dt_est_half = dt_est;
          const int rej = dt_est < dt;
          s->rejected = rej;
          if (rej) s->dt_ctl = dt_est > 0.0 ? 0.85 * dt_est : 0.5 * dt;
          else if (s->dt_ctl > 0.0) s->dt_ctl *= 1.02;
        } else {
          s->dt_est = dt_est;
          double dt = a.fixed_dt;
          if (!(dt > 0.0)) {
            dt = fmin(dt_est, s->t_end - s->t);
            if (a.ctl == 1 && s->dt_ctl > 0.0) dt = fmin(dt, s->dt_ctl);
          }
          if (!(dt > 0.0)) dt = 0.0;
          s->dt = dt;
          if (a.ctl == 1) s->rejected = 0;
        }
      }
    }
  }

  // ===== force product F.u (row b1), element part -> E-vector =============
  // smem: tab | f[DIM][CX][NQ] | S | y[CX][ND] | ul[NB][NL] | uq[NB][NQ]
  static constexpr int F_S = max3(grad_scratch<DIM, D, Q>(CX), interp_scratch<DIM, L, Q>(NB), 0);
  static constexpr size_t force_smem() {
    return sizeof(double) * (TAB + DIM * CX * NQ + F_S + CX * ND + NB * NL + NB * NQ);
  }
  static __device__ __forceinline__ void body_force(const ForceArgs &a, int e0) {
    extern __shared__ double sm[];
    double *st = sm, *f = st + TAB, *S = f + DIM * CX * NQ, *y = S + F_S, *ul = y + CX * ND, *uq = ul + NB * NL;
    const MeshDesc &m = a.mesh;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    // D[e][c*DIM+l][q] -> f[l][b*DIM+c][q]  (one contiguous global block per CTA)
    for (int k = threadIdx.x; k < NB * DIM * DIM * NQ; k += blockDim.x) {
      const int q = k % NQ, r = (k / NQ) % (DIM * DIM), b = k / (NQ * DIM * DIM);
      const int c = r / DIM, l = r % DIM;
      f[(l * CX + b * DIM + c) * NQ + q] = b < nb ? a.D[(size_t)e0 * DIM * DIM * NQ + k] : 0.0;
    }
    if (a.u) {
      for (int k = threadIdx.x; k < NB * NL; k += blockDim.x)
        ul[k] = k / NL < nb ? a.u[(size_t)e0 * NL + k] : 0.0;
      __syncthreads();
      interp<DIM, L, Q, NB>(ul, uq, S, st + oBl);
      for (int k = threadIdx.x; k < DIM * CX * NQ; k += blockDim.x) {
        const int q = k % NQ, b = ((k / NQ) % CX) / DIM;
        f[k] *= uq[b * NQ + q];
      }
    }
    __syncthreads();
    grad_ref_t<DIM, D, Q, CX>(f, y, S, st + oBt, st + oGt);
    for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x) a.evec[(size_t)e0 * DIM * ND + k] = y[k];
  }

  // ===== transposed force product F^T v (row b2), optionally fused with the
  // TG-2D energy source, the energy solve M_E^{-1} (row c3) and the e update (row c4).
  // smem: tab | u[CX][ND] | xu[CX][ND] | S | g[DIM][CX][NQ] | xq[CX][NQ] | sq[NB][NQ] | out[NB][NL] | red
  static constexpr int FT_S = max3(grad_scratch<DIM, D, Q>(CX), interp_scratch<DIM, D, Q>(CX),
                                   interp_scratch<DIM, Q, L>(NB));
  static constexpr size_t force_t_smem() {
    return sizeof(double) * (TAB + 2 * CX * ND + FT_S + DIM * CX * NQ + CX * NQ + NB * NQ + NB * NL + RED);
  }
  static __device__ __forceinline__ void body_force_t(const ForceTArgs &a, int e0) {
    if (a.skip && *a.skip) return;   // uniform over the grid: the step was rejected
    extern __shared__ double sm[];
    double *st = sm, *u = st + TAB, *xu = u + CX * ND, *S = xu + CX * ND, *g = S + FT_S;
    double *xq = g + DIM * CX * NQ, *sq = xq + CX * NQ, *out = sq + NB * NQ, *red = out + NB * NL;
    const MeshDesc &m = a.mesh;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    gather_elem(u, a.v, DIM, m, e0, nb);
    if (a.src_x) gather_elem(xu, a.src_x, DIM, m, e0, nb);
    __syncthreads();
    grad_ref<DIM, D, Q, CX>(u, g, S, st + oB, st + oG);
    if (a.src_x) interp<DIM, D, Q, CX>(xu, xq, S, st + oB);   // positions at qpoints
    double src_sum = 0.0;
    for (int k = threadIdx.x; k < NB * NQ; k += blockDim.x) {
      const int b = k / NQ, q = k % NQ;
      double s = 0.0;
      if (b < nb) {
        const size_t base = (size_t)(e0 + b) * DIM * DIM * NQ + q;
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
          for (int l = 0; l < DIM; ++l)
            s = fma(a.D[base + (size_t)(c * DIM + l) * NQ], g[(l * CX + b * DIM + c) * NQ + q], s);
        if (a.src_x) {
          // 2D Taylor-Green internal-energy source Q(x), weighted by omega rho0 detJ0
          const double X = xq[(b * DIM + 0) * NQ + q], Y = xq[(b * DIM + 1) * NQ + q];
          const double pi = 3.141592653589793;
          const double Qs = (3.0 * pi / 8.0) * (cos(3.0 * pi * X) * cos(pi * Y) - cos(pi * X) * cos(3.0 * pi * Y));
          const double sv = a.mq[(size_t)(e0 + b) * NQ + q] * Qs;
          s += sv;
          src_sum += sv;
        }
      }
      sq[k] = s;
    }
    __syncthreads();
    interp<DIM, Q, L, NB>(sq, out, S, st + oBlt);   // sum_q phi_j(q) s_q
    if (!a.me_inv) {
      for (int k = threadIdx.x; k < nb * NL; k += blockDim.x) a.out[(size_t)e0 * NL + k] = out[k];
    } else {
      const double coef = a.coef * *a.dt;
      for (int k = threadIdx.x; k < nb * NL; k += blockDim.x) {
        const int b = k / NL, j = k % NL;
        double s;
        apply_me_inv(a.me_inv, out + b * NL, e0 + b, j, s);
        const size_t idx = (size_t)e0 * NL + k;
        a.out[idx] = fma(coef, s, a.e_base[idx]);
      }
    }
    if (!a.src_sum) return;
    double v1[1] = {src_sum};
    bsum<1>(v1, red);
    __shared__ int s_last;
    if (threadIdx.x == 0) {
      a.partials[blockIdx.x] = v1[0];
      __threadfence();
      s_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || threadIdx.x >= 32) return;
    __threadfence();
    double sacc = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) sacc += ((volatile double *)a.partials)[i];
    sacc = warp_sum(sacc);
    if (threadIdx.x == 0) {
      *a.counter = 0u;
      *a.src_sum = sacc * *a.dt;
    }
  }

  // ===== PA mass action (row c1), element part =============================
  // smem: tab | u[CX][ND] | S | uq[CX][NQ] | y[CX][ND] | red
  static constexpr int M_S = max3(interp_scratch<DIM, D, Q>(CX), interp_scratch<DIM, Q, D>(CX), 0);
  static constexpr size_t mass_smem() {
    return sizeof(double) * (TAB + CX * ND + M_S + CX * NQ + CX * ND + RED);
  }
  // y_e = B^T diag(mq) B u_e for the DIM components of NB elements
  static __device__ __forceinline__ void mass_elem(const double *st, const double *u, double *S, double *uq,
                                                   double *y, const double *__restrict__ mq, int e0, int nb) {
    interp<DIM, D, Q, CX>(u, uq, S, st + oB);
    for (int k = threadIdx.x; k < CX * NQ; k += blockDim.x) {
      const int q = k % NQ, b = (k / NQ) / DIM;
      uq[k] *= b < nb ? mq[(size_t)(e0 + b) * NQ + q] : 0.0;
    }
    __syncthreads();
    interp<DIM, Q, D, CX>(uq, y, S, st + oBt);
  }
  static __device__ __forceinline__ void body_mass(const MassArgs &a, int e0) {
    extern __shared__ double sm[];
    double *st = sm, *u = st + TAB, *S = u + CX * ND, *uq = S + M_S, *y = uq + CX * NQ;
    const MeshDesc &m = a.mesh;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    gather_elem(u, a.x, DIM, m, e0, nb);
    __syncthreads();
    mass_elem(st, u, S, uq, y, a.mq, e0, nb);
    for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x) a.evec[(size_t)e0 * DIM * ND + k] = y[k];
  }

  // ===== Jacobi-PCG on the PA mass operator (row c2), one persistent launch
  // CTAs of the persistent solvers are CGM times larger than the element
  // kernels' (fewer blocks make the grid barriers cheaper).
  static constexpr int CGM = 2 * THREADS <= 1024 ? 2 : 1;
  static constexpr int NBC = NB * CGM;          // elements per solver CTA and batch
  static constexpr int TC = THREADS * CGM;      // threads per solver CTA
  static constexpr int CXC = NBC * DIM;
  // FP64 solver CTAs per SM the register allocation must allow (launch bounds of
  // k_cg): two, as the solver has been measured with (barriers and memory round
  // trips bound it as much as FP64 work); 2D Q3 runs one CTA per SM with more
  // registers, also as measured. Without the bound ptxas may take 98 registers at
  // Q3/Q4 and halve the occupancy.
  static constexpr int CG_MINB = DIM == 2 && P == 3 ? 1 : 2;
  // the same for the precision form's solver (k_cg_ir), as measured: two CTAs per
  // SM up to p = 2 and at 3D Q3, one at 2D Q3 and at Q4 (registers)
  static constexpr int CGIR_MINB = P <= 2 || (DIM == 3 && P == 3) ? 2 : 1;
  static constexpr int MC_S = max3(interp_scratch<DIM, D, Q>(CXC), interp_scratch<DIM, Q, D>(CXC), 0);

  // E-vector of M u for one batch: y = B^T diag(mq) B u (CXC tensors), T arithmetic.
  template <typename T>
  static __device__ __forceinline__ void batch_matvec(const T *tb, const T *tbt, const T *u, T *S, T *uq, T *y,
                                                      const T *__restrict__ mq, int e0, int nb) {
    interp<DIM, D, Q, CXC>(u, uq, S, tb);
    for (int k = threadIdx.x; k < CXC * NQ; k += blockDim.x) {
      const int q = k % NQ, b = (k / NQ) / DIM;
      uq[k] *= b < nb ? mq[(size_t)(e0 + b) * NQ + q] : (T)0;
    }
    __syncthreads();
    interp<DIM, Q, D, CXC>(uq, y, S, tbt);
  }

  // The same product with the batch's mass data loaded into registers by the caller
  // (load_mq) before its gather, so that those loads overlap the gather and the
  // first contraction instead of following them. Value k of the batch belongs to
  // thread k mod blockDim.x; MQT_C values per thread cover the batch only when
  // blockDim.x >= TC, which the callers check (the tensor-core solver runs this
  // family's FP64 sweeps with a different block size).
  static constexpr int MQT_C = (CXC * NQ + TC - 1) / TC;
  template <typename T>
  static __device__ __forceinline__ void load_mq(const T *__restrict__ mq, int e0, int nb, T (&r)[MQT_C]) {
#pragma unroll
    for (int j = 0; j < MQT_C; ++j) {
      const int k = threadIdx.x + j * blockDim.x;
      const int q = k % NQ, b = (k / NQ) / DIM;
      r[j] = (k < CXC * NQ && b < nb) ? mq[(size_t)(e0 + b) * NQ + q] : (T)0;
    }
  }
  template <typename T>
  static __device__ __forceinline__ void batch_matvec_r(const T *tb, const T *tbt, const T *u, T *S, T *uq, T *y,
                                                        const T (&r)[MQT_C]) {
    interp<DIM, D, Q, CXC>(u, uq, S, tb);
#pragma unroll
    for (int j = 0; j < MQT_C; ++j) {
      const int k = threadIdx.x + j * blockDim.x;
      if (k < CXC * NQ) uq[k] *= r[j];
    }
    __syncthreads();
    interp<DIM, Q, D, CXC>(uq, y, S, tbt);
  }

  // Search-direction value at a node: p_new = invdiag*(r - alpha q) + beta p (MODE 2),
  // p0 = invdiag*r (MODE 1), invdiag*r + beta p (MODE 3), z + beta p with z = invdiag*r
  // passed as x (MODE 4), or the masked vector x (MODE 0).
  template <int MODE, typename T>
  static __device__ __forceinline__ T dir_value(int gi, const T *__restrict__ idv, const T *x, const T *r,
                                                const T *q, const T *p, T alpha, T beta) {
    if (MODE == 4) return fma(beta, p[gi], x[gi]);   // x holds z = invdiag r
    const T idg = idv[gi];
    if (MODE == 0) return idg != (T)0 ? x[gi] : (T)0;
    if (MODE == 1) return idg * r[gi];
    if (MODE == 3) return fma(beta, p[gi], idg * r[gi]);
    return fma(beta, p[gi], idg * fma(-alpha, q[gi], r[gi]));
  }

  // One sweep over all element batches: E-vector of M times the MODE vector.
  // With dot != nullptr each thread also accumulates sum_e u_e . (M_e u_e) over
  // the values it stores: the energy u^T M u of the swept vector, element by element.
  template <int MODE, typename T>
  static __device__ __forceinline__ void sweep_matvec(const MeshDesc &m, int *eb, const T *tb, const T *tbt, T *u,
                                                      T *S, T *uq, T *y, const T *mq, const T *idv, const T *x,
                                                      const T *r, const T *q, const T *p, T alpha, T beta,
                                                      T *evec, T *dot = nullptr) {
    const int nbatch = (m.ne + NBC - 1) / NBC;
    for (int bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
      const int e0 = bt * NBC, nb = min(NBC, m.ne - e0);
      const bool pre = blockDim.x >= TC;   // block-uniform
      T mqr[MQT_C];   // mass data first: the loads overlap the gather below
      if (pre) load_mq<T>(mq, e0, nb, mqr);
      if (threadIdx.x < nb) eb[threadIdx.x] = h1_base<DIM, D>(m, e0 + threadIdx.x);
      __syncthreads();
      for (int k = threadIdx.x; k < CXC * ND; k += blockDim.x) {
        const int i = k % ND, bc = k / ND, c = bc % DIM, b = bc / DIM;
        T val = 0;
        if (b < nb) val = dir_value<MODE, T>(c * m.nh1 + eb[b] + h1_local<DIM, D>(m, i), idv, x, r, q, p, alpha, beta);
        u[k] = val;
      }
      __syncthreads();
      if (pre) batch_matvec_r<T>(tb, tbt, u, S, uq, y, mqr);
      else batch_matvec<T>(tb, tbt, u, S, uq, y, mq, e0, nb);
      if (dot) {
        T d = *dot;
        for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x) {
          const T yk = y[k];
          evec[(size_t)e0 * DIM * ND + k] = yk;
          d = fma(u[k], yk, d);
        }
        *dot = d;
      } else {
        for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x) evec[(size_t)e0 * DIM * ND + k] = y[k];
      }
      __syncthreads();
    }
  }

  // FP32 sweeps of the precision form use their own, larger element batches
  // (FP32 arithmetic is cheap, so batch latency dominates): as many elements as
  // fit in ~96 KB of shared memory (~64 KB at 3D Q2), at most 64.
  static constexpr int PER_ELEM_F = 2 * DIM * ND + DIM * NQ +
                                    (interp_scratch<DIM, D, Q>(DIM) > interp_scratch<DIM, Q, D>(DIM)
                                         ? interp_scratch<DIM, D, Q>(DIM) : interp_scratch<DIM, Q, D>(DIM));
#ifndef LH_NBF_FLOATS
#define LH_NBF_FLOATS 24000
#endif
#ifndef LH_NBF_FLOATS_3D_Q2
#define LH_NBF_FLOATS_3D_Q2 16000
#endif
  // 3D Q2 takes a smaller budget (32 elements per batch instead of 48): measured
  // 9 % faster per FP32 step at 24^3 (1.5 batches per CTA, more L1 beside the
  // smaller shared-memory footprint), 3 % slower at 32^3; every other family keeps
  // 24,000 floats (both directions measured slower at Q3 and Q4)
  static constexpr int NBF_BUDGET = DIM == 3 && P == 2 ? LH_NBF_FLOATS_3D_Q2 : LH_NBF_FLOATS;
  static constexpr int NBF_RAW = NBF_BUDGET / PER_ELEM_F;
  static constexpr int NBF = NBF_RAW < 1 ? 1 : (NBF_RAW > 64 ? 64 : NBF_RAW);
  static constexpr int CXF = NBF * DIM;
  static constexpr int MF_S = max3(interp_scratch<DIM, D, Q>(CXF), interp_scratch<DIM, Q, D>(CXF), 0);
  static constexpr int NB_EB = NBF > NBC ? NBF : NBC;   // size of the per-batch base-node table

  template <int MODE>
  static __device__ __forceinline__ void sweep_matvec_f(const MeshDesc &m, int *eb, const float *tb,
                                                        const float *tbt, float *u, float *S, float *uq, float *y,
                                                        const float *mq, const float *idv, const float *x,
                                                        const float *r, const float *q, const float *p, float alpha,
                                                        float beta, float *evec, float &dot) {
    const int nbatch = (m.ne + NBF - 1) / NBF;
    constexpr int MQT = (CXF * NQ + TC - 1) / TC;   // mass-data values per thread (blockDim == TC)
    constexpr bool kPrefetch = MQT <= 16;
    if constexpr (P >= 4) {
      // high orders (one CTA per SM, many batches per CTA): software-pipelined gather.
      // The next batch's values are loaded into registers right after this batch's
      // have been stored, so their latency overlaps this batch's contractions.
      constexpr int GV = (CXF * ND + TC - 1) / TC;
      float nxt[GV];
      auto gather_regs = [&](int nbg) {
#pragma unroll
        for (int v = 0; v < GV; ++v) {
          const int k = threadIdx.x + v * TC;
          const int i = k % ND, bc = k / ND, c = bc % DIM, b = bc / DIM;
          nxt[v] = (k < CXF * ND && b < nbg)
                       ? dir_value<MODE, float>(c * m.nh1 + eb[b] + h1_local<DIM, D>(m, i), idv, x, r, q, p, alpha,
                                                beta)
                       : 0.0f;
        }
      };
      int bt = blockIdx.x;
      if (bt < nbatch) {
        const int nb = min(NBF, m.ne - bt * NBF);
        if (threadIdx.x < nb) eb[threadIdx.x] = h1_base<DIM, D>(m, bt * NBF + threadIdx.x);
        __syncthreads();
        gather_regs(nb);
        // every warp has read eb before the loop overwrites it with the next batch's
        // base nodes (one barrier per sweep; no measurable cost at 32^3 Q4)
        __syncthreads();
      }
      for (; bt < nbatch; bt += gridDim.x) {
        const int e0 = bt * NBF, nb = min(NBF, m.ne - e0);
        float mqr[kPrefetch ? MQT : 1];
        if constexpr (kPrefetch) {
#pragma unroll
          for (int j = 0; j < MQT; ++j) {
            const int k = threadIdx.x + j * TC;
            const int qq = k % NQ, b = (k / NQ) / DIM;
            mqr[j] = (k < CXF * NQ && b < nb) ? mq[(size_t)(e0 + b) * NQ + qq] : 0.0f;
          }
        }
#pragma unroll
        for (int v = 0; v < GV; ++v) {
          const int k = threadIdx.x + v * TC;
          if (k < CXF * ND) u[k] = nxt[v];
        }
        // base nodes of the next batch (every earlier reader of eb is past a barrier)
        const int btn = bt + gridDim.x;
        const int nbn = btn < nbatch ? min(NBF, m.ne - btn * NBF) : 0;
        if (threadIdx.x < nbn) eb[threadIdx.x] = h1_base<DIM, D>(m, btn * NBF + threadIdx.x);
        __syncthreads();
        if (nbn > 0) gather_regs(nbn);
        interp_p<DIM, D, Q, CXF>(u, uq, S, tb);
        if constexpr (kPrefetch) {
#pragma unroll
          for (int j = 0; j < MQT; ++j) {
            const int k = threadIdx.x + j * TC;
            if (k < CXF * NQ) uq[k] *= mqr[j];
          }
        } else {
          for (int k = threadIdx.x; k < CXF * NQ; k += blockDim.x) {
            const int qq = k % NQ, b = (k / NQ) / DIM;
            uq[k] *= b < nb ? mq[(size_t)(e0 + b) * NQ + qq] : 0.0f;
          }
        }
        __syncthreads();
        interp_p<DIM, Q, D, CXF>(uq, y, S, tbt);
        for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x) {
          const float yk = y[k];
          evec[(size_t)e0 * DIM * ND + k] = yk;
          dot = fmaf(u[k], yk, dot);
        }
        __syncthreads();
      }
      return;
    }
    for (int bt = blockIdx.x; bt < nbatch; bt += gridDim.x) {
      const int e0 = bt * NBF, nb = min(NBF, m.ne - e0);
      // issue this batch's mass-data loads first: they are needed only after the
      // first contraction stages, so their latency overlaps the gather and stages
      // (only while the prefetch array is small: more registers would cost occupancy)
      float mqr[kPrefetch ? MQT : 1];
      if constexpr (kPrefetch) {
#pragma unroll
        for (int j = 0; j < MQT; ++j) {
          const int k = threadIdx.x + j * TC;
          const int qq = k % NQ, b = (k / NQ) / DIM;
          mqr[j] = (k < CXF * NQ && b < nb) ? mq[(size_t)(e0 + b) * NQ + qq] : 0.0f;
        }
      }
      if (threadIdx.x < nb) eb[threadIdx.x] = h1_base<DIM, D>(m, e0 + threadIdx.x);
      __syncthreads();
      // gather: GU values per pass, every global load of the pass issued before the
      // shared-memory stores (a store through a generic pointer would otherwise hold
      // the next value's loads back)
      constexpr int GU = 4;
      for (int k0 = threadIdx.x; k0 < CXF * ND; k0 += GU * blockDim.x) {
        float val[GU];
#pragma unroll
        for (int uix = 0; uix < GU; ++uix) {
          const int k = k0 + uix * blockDim.x;
          const int i = k % ND, bc = k / ND, c = bc % DIM, b = bc / DIM;
          val[uix] = (k < CXF * ND && b < nb)
                         ? dir_value<MODE, float>(c * m.nh1 + eb[b] + h1_local<DIM, D>(m, i), idv, x, r, q, p, alpha,
                                                  beta)
                         : 0.0f;
        }
#pragma unroll
        for (int uix = 0; uix < GU; ++uix) {
          const int k = k0 + uix * blockDim.x;
          if (k < CXF * ND) u[k] = val[uix];
        }
      }
      __syncthreads();
      interp_p<DIM, D, Q, CXF>(u, uq, S, tb);
      if constexpr (kPrefetch) {
#pragma unroll
        for (int j = 0; j < MQT; ++j) {
          const int k = threadIdx.x + j * TC;
          if (k < CXF * NQ) uq[k] *= mqr[j];
        }
      } else {
        for (int k = threadIdx.x; k < CXF * NQ; k += blockDim.x) {
          const int qq = k % NQ, b = (k / NQ) / DIM;
          uq[k] *= b < nb ? mq[(size_t)(e0 + b) * NQ + qq] : 0.0f;
        }
      }
      __syncthreads();
      interp_p<DIM, Q, D, CXF>(uq, y, S, tbt);
      for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x) {
        const float yk = y[k];
        evec[(size_t)e0 * DIM * ND + k] = yk;
        dot = fmaf(u[k], yk, dot);
      }
      __syncthreads();
    }
  }

  static constexpr size_t cg_smem() { return sizeof(double) * (TAB + CXC * ND + MC_S + CXC * NQ + CXC * ND + RED); }
  // Jacobi PCG with the standard recurrences and two grid barriers per
  // iteration: p.Mp is summed element by element inside the element sweep
  // (u_e . M_e u_e), so alpha is known after the first barrier and a single node
  // sweep gathers q, updates p, x, r, z and forms r.r and r.z.
  static __device__ __forceinline__ void body_cg(CgArgs a) {
    extern __shared__ double sm[];
    double *st = sm, *u = st + TAB, *S = u + CXC * ND, *uq = S + MC_S, *y = uq + CXC * NQ, *red = y + CXC * ND;
    __shared__ double s_sc[8];
    __shared__ int s_eb[NBC];
    const MeshDesc &m = a.mesh;
    const int G = gridDim.x;
    const int nh1 = m.nh1;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gstride = G * blockDim.x;
    GridBarrier *bar = (GridBarrier *)a.bar;
    unsigned long long nbar = 0;
    auto sync = [&]() { ++nbar; return grid_sync(bar, nbar * (unsigned long long)G, a.status); };
    load_tab(st, a.tab);
    __syncthreads();
    const double *tb = st + oB, *tbt = st + oBt;
    auto finish = [&](int iters, int status, double rr, double bb) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double bn = sqrt(bb);
        const double rel = bn > 0.0 ? sqrt(rr) / bn : 0.0;
        if (a.info) {
          a.info->iters = iters;
          a.info->status = status;
          a.info->rel_res = rel;
          a.info->b_norm = bn;
          a.info->refinements = 0;
        }
        if (a.iters_out) *a.iters_out = iters;
        if (a.relres_out) *a.relres_out = rel;
        if (status) latch_status(a.status, status);
      }
    };
    // ---- init: r0 = b - A x0 on free DOFs; x0 = 0 on constrained DOFs
    sweep_matvec<0, double>(m, s_eb, tb, tbt, u, S, uq, y, a.mq, a.invdiag, a.x, a.r, a.ap, a.p, 0.0, 0.0, a.evec);
    if (!sync()) { finish(0, kStatusTimeout, 0.0, 0.0); return; }
    {
      double acc[3] = {0.0, 0.0, 0.0};   // b.b, r.r, r.z
      for (int g = gtid; g < nh1; g += gstride) {
        int off[1 << DIM];
        const int n = node_copies<DIM, D>(m, g, DIM, off);
        for (int c = 0; c < DIM; ++c) {
          const int k = c * nh1 + g;
          const double idg = a.invdiag[k];
          double rv = 0.0;
          if (idg != 0.0) {
            double ax = a.evec[off[0] + c * ND];
            for (int j = 1; j < n; ++j) ax += a.evec[off[j] + c * ND];
            const double bv = a.b[k];
            rv = bv - ax;
            acc[0] = fma(bv, bv, acc[0]);
            acc[1] = fma(rv, rv, acc[1]);
            acc[2] = fma(rv * idg, rv, acc[2]);
          } else {
            a.x[k] = 0.0;
          }
          a.r[k] = rv;
          a.z[k] = rv * idg;
          a.p[k] = 0.0;
          a.ap[k] = 0.0;
        }
      }
      bsum<3>(acc, red);
      if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) a.partials[(size_t)q * G + blockIdx.x] = acc[q];
    }
    if (!sync()) { finish(0, kStatusTimeout, 0.0, 0.0); return; }
    if (threadIdx.x < 32) {
      double v[3];
      for (int k = 0; k < 3; ++k) v[k] = warp_sum_partials(a.partials + (size_t)k * G, G);
      if (threadIdx.x == 0) { s_sc[0] = v[0]; s_sc[1] = v[1]; s_sc[2] = v[2]; }
    }
    __syncthreads();
    const double bb = s_sc[0];
    const double tol2 = a.tol * a.tol * bb;
    double rr = s_sc[1], rz = s_sc[2], rz_old = rz;
    if (bb == 0.0) {
      for (int k = gtid; k < DIM * nh1; k += gstride) a.x[k] = 0.0;
      finish(0, 0, 0.0, 0.0);
      return;
    }
    int it = 0;
    for (;;) {
      if (rr <= tol2) { finish(it, 0, rr, bb); return; }
      if (it >= a.max_it) { finish(it, 5, rr, bb); return; }
      if (threadIdx.x == 0) s_sc[5] = it == 0 ? 0.0 : rz / rz_old;   // beta, once per block
      __syncthreads();
      const double beta = s_sc[5];
      rz_old = rz;
      // E-vector of M p_new, p_new = z + beta p (z = invdiag r, stored by the r update),
      // and p_new . M p_new summed element by element (p_new = 0 on constrained DOFs)
      {
        double pq = 0.0;
        sweep_matvec<4, double>(m, s_eb, tb, tbt, u, S, uq, y, a.mq, a.invdiag, a.z, a.r, a.ap, a.p, 0.0, beta,
                                a.evec, &pq);
        double acc[1] = {pq};
        bsum<1>(acc, red);
        if (threadIdx.x == 0) a.partials[(size_t)3 * G + blockIdx.x] = acc[0];
      }
      if (!sync()) { finish(it, kStatusTimeout, rr, bb); return; }
      if (threadIdx.x < 32) {
        const double v = warp_sum_partials(a.partials + (size_t)3 * G, G);
        if (threadIdx.x == 0) s_sc[4] = rz / v;   // alpha, once per block
      }
      __syncthreads();
      const double alpha = s_sc[4];
      {  // one node sweep: q = M p_new gathered, p = p_new, x += alpha p, r -= alpha q,
         // z = invdiag r, r.r and r.z; one (node, component) per work item, its
         // copies located through the node-copy table, every load issued first
        double acc[2] = {0.0, 0.0};
        // one contiguous share of equal size per block: the sweep is FP64-issue
        // bound per SM, and a grid-stride split gives the first blocks (2 of 3 SMs
        // at 24^3 Q2) one item more per thread (measured 1.35 % per step; the
        // latency-bound FP32 node sweeps keep the grid-stride split, measured faster)
        int k0, k1;
        block_chunk(DIM * nh1, k0, k1);
        for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) {
          const int c = DIM == 2 ? (k >= nh1 ? 1 : 0) : (k >= 2 * nh1 ? 2 : (k >= nh1 ? 1 : 0));
          const int g = k - c * nh1;
          int off[1 << DIM];
          node_table_row<DIM>(a.ncopy, g, off);
          const double idg = __ldg(a.invdiag + k);
          const double pv = a.p[k], zv = a.z[k], xv = a.x[k], rv = a.r[k];
          double ev[1 << DIM];
#pragma unroll
          for (int j = 0; j < (1 << DIM); ++j) ev[j] = off[j] >= 0 ? a.evec[off[j] + c * ND] : 0.0;
          double qv = ev[0];
#pragma unroll
          for (int j = 1; j < (1 << DIM); ++j)
            if (off[j] >= 0) qv += ev[j];
          // constrained DOFs (Jacobi inverse exactly +0) keep p = r = z = 0; the test
          // reads the bit pattern, so it runs on the integer pipe and leaves the FP64
          // pipe, which bounds this sweep, to the arithmetic
          if (__double_as_longlong(idg) != 0LL) {
            const double pn = fma(beta, pv, zv);
            const double r2 = fma(-alpha, qv, rv);
            const double z2 = r2 * idg;
            a.p[k] = pn;
            a.x[k] = fma(alpha, pn, xv);
            a.r[k] = r2;
            a.z[k] = z2;
            acc[0] = fma(r2, r2, acc[0]);
            acc[1] = fma(z2, r2, acc[1]);
          }
        }
        bsum<2>(acc, red);
        if (threadIdx.x == 0) {
          a.partials[(size_t)1 * G + blockIdx.x] = acc[0];
          a.partials[(size_t)2 * G + blockIdx.x] = acc[1];
        }
      }
      if (!sync()) { finish(it, kStatusTimeout, rr, bb); return; }
      static_assert(TC >= 64, "the solver's final sums take two warps");
      if (threadIdx.x < 64) {   // r.r on warp 0, r.z on warp 1, side by side
        const int w = threadIdx.x >> 5;
        const double v = warp_sum_partials(a.partials + (size_t)(1 + w) * G, G);
        if ((threadIdx.x & 31) == 0) s_sc[1 + w] = v;
      }
      __syncthreads();
      rr = s_sc[1];
      rz = s_sc[2];
      ++it;
    }
  }

  // ===== precision form: FP32 inner PCG under FP64 iterative refinement ===
  // Outer (FP64): r = b - M x, ||r|| check, x += d. Inner (FP32): the same
  // two-barrier Jacobi PCG on M d = r from d = 0 to a relative residual
  // inner_tol, with FP32 tables, mass data, vectors, element vectors, partial
  // sums and scalars.
  static constexpr int IR_F = 2 * Q * D + CXF * ND + MF_S + CXF * NQ + CXF * ND;   // floats
  static constexpr int IR_D = CXC * ND + MC_S + CXC * NQ + CXC * ND;               // doubles
  static constexpr int IR_R = (IR_F + 1) / 2 > IR_D ? (IR_F + 1) / 2 : IR_D;
  static constexpr size_t cg_ir_smem() { return sizeof(double) * (TAB + IR_R + RED); }
  static __device__ __forceinline__ void body_cg_ir(CgIrArgs a) {
    extern __shared__ double sm[];
    double *st = sm, *R = st + TAB, *red = R + IR_R;
    double *u = R, *S = u + CXC * ND, *uq = S + MC_S, *y = uq + CXC * NQ;                 // FP64 view
    float *tb = (float *)R, *tbt = tb + Q * D, *uf = tbt + Q * D, *Sf = uf + CXF * ND;    // FP32 view
    float *uqf = Sf + MF_S, *yf = uqf + CXF * NQ;
    __shared__ int s_eb[NB_EB];
    load_tab(st, a.tab);
    __syncthreads();
    cg_ir_core<false>(
        a, st, u, S, uq, y, red, s_eb,
        [&]() {   // FP32 copies of the 1D tables (the FP64 sweep reuses this space)
          for (int k = threadIdx.x; k < 2 * Q * D; k += blockDim.x)
            tb[k] = (float)(k < Q * D ? st[oB + k] : st[oBt + k - Q * D]);
          __syncthreads();
        },
        [&](float beta, float &pq) {
          sweep_matvec_f<4>(a.mesh, s_eb, tb, tbt, uf, Sf, uqf, yf, a.mq32, a.invdiag32, a.z32, a.r32, a.ap32,
                            a.p32, 0.0f, beta, a.evec32, pq);
          return true;
        });
  }

  // The refinement loop shared by the CUDA-core (body_cg_ir) and tensor-core
  // (lh_tc.cuh) inner solvers: inner_begin() runs before each inner solve,
  // inner_sweep(beta, pq) writes the FP32 E-vector of M p_new and adds this
  // thread's share of p_new . M p_new to pq (false: a bounded
  // device wait gave up). st/u/S/uq/y: FP64 sweep space; RELOAD_TAB: the
  // FP64 tables share space with the inner sweep and are reloaded per refinement.
  template <bool RELOAD_TAB, class Begin, class Sweep>
  static __device__ __forceinline__ void cg_ir_core(const CgIrArgs &a, double *st, double *u, double *S, double *uq,
                                                    double *y, double *red, int *s_eb, Begin &&inner_begin,
                                                    Sweep &&inner_sweep) {
    float *redf = (float *)red;
    __shared__ double s_sc[4];
    __shared__ float s_f[4];
    const MeshDesc &m = a.mesh;
    const int G = gridDim.x;
    const int nh1 = m.nh1;
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int gstride = G * blockDim.x;
    float *pf = (float *)(a.partials + (size_t)4 * G);   // FP32 partial rows: 5 rows of G floats
    GridBarrier *bar = (GridBarrier *)a.bar;
    unsigned long long nbar = 0;
    auto sync = [&]() { ++nbar; return grid_sync(bar, nbar * (unsigned long long)G, a.status); };
    int outer = 0;
    auto finish = [&](int iters, int status, double rr, double bb) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double bn = sqrt(bb);
        const double rel = bn > 0.0 ? sqrt(rr) / bn : 0.0;
        if (a.info) {
          a.info->iters = iters;
          a.info->status = status;
          a.info->rel_res = rel;
          a.info->b_norm = bn;
          a.info->refinements = outer;
        }
        if (a.iters_out) *a.iters_out = iters;
        if (a.relres_out) *a.relres_out = rel;
        if (status) latch_status(a.status, status);
      }
    };
    // FP32 block sums of the N <= 5 values of v into thread 0's v (warp shuffles).
    auto block_sum_f = [&](auto &v) {
      constexpr int N = (int)(sizeof(v) / sizeof(v[0]));
      static_assert(N <= 5, "reduction scratch holds five values");
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
      for (int k = 0; k < N; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
      __syncthreads();
      if (lane == 0)
        for (int k = 0; k < N; ++k) redf[k * 32 + warp] = v[k];
      __syncthreads();
      if (warp == 0)
        for (int k = 0; k < N; ++k) {
          float t = lane < nw ? redf[k * 32 + lane] : 0.0f;
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          v[k] = t;
        }
    };

    double bb = -1.0;
    int inner_total = 0;
    for (;; ++outer) {
      if constexpr (RELOAD_TAB) {
        load_tab(st, a.tab);
        __syncthreads();
      }
      // ---- O-A: FP64 E-vector of M x (x masked to the free DOFs)
      sweep_matvec<0, double>(m, s_eb, st + oB, st + oBt, u, S, uq, y, a.mq, a.invdiag, a.x, a.x, a.x, a.x, 0.0,
                              0.0, a.evec);
      if (!sync()) { finish(inner_total, kStatusTimeout, 0.0, 0.0); return; }
      // ---- O-B: FP64 residual and its FP32 copy; inner start d = 0
      {
        double acc[2] = {0.0, 0.0};   // b.b, r.r
        float accf[2] = {0, 0};   // r32.r32, r32.z32
        for (int g = gtid; g < nh1; g += gstride) {
          int off[1 << DIM];
          const int n = node_copies<DIM, D>(m, g, DIM, off);
          for (int c = 0; c < DIM; ++c) {
            const int k = c * nh1 + g;
            float rf = 0.0f;
            if (a.invdiag[k] != 0.0) {
              double ax = a.evec[off[0] + c * ND];
              for (int j = 1; j < n; ++j) ax += a.evec[off[j] + c * ND];
              const double bv = a.b[k];
              const double rv = bv - ax;
              if (outer == 0) acc[0] = fma(bv, bv, acc[0]);
              acc[1] = fma(rv, rv, acc[1]);
              rf = (float)rv;
              accf[0] = fmaf(rf, rf, accf[0]);
              accf[1] = fmaf(rf * a.invdiag32[k], rf, accf[1]);
            } else {
              a.x[k] = 0.0;
            }
            a.r32[k] = rf;
            a.z32[k] = rf * a.invdiag32[k];
            a.d32[k] = 0.0f;
            a.p32[k] = 0.0f;
            a.ap32[k] = 0.0f;
          }
        }
        bsum<2>(acc, red);
        if (threadIdx.x == 0) {
          a.partials[blockIdx.x] = acc[0];
          a.partials[(size_t)G + blockIdx.x] = acc[1];
        }
        block_sum_f(accf);
        if (threadIdx.x == 0) {
          pf[blockIdx.x] = accf[0];
          pf[(size_t)G + blockIdx.x] = accf[1];
        }
      }
      if (!sync()) { finish(inner_total, kStatusTimeout, 0.0, 0.0); return; }
      if (threadIdx.x < 32) {
        const double s0 = outer == 0 ? warp_sum_partials(a.partials, G) : 0.0;
        const double s1 = warp_sum_partials(a.partials + G, G);
        float f[2];
        for (int k2 = 0; k2 < 2; ++k2) f[k2] = warp_sum_partials_f(pf + (size_t)k2 * G, G);
        if (threadIdx.x == 0) { s_sc[0] = s0; s_sc[1] = s1; s_f[0] = f[0]; s_f[1] = f[1]; }
      }
      __syncthreads();
      if (outer == 0) bb = s_sc[0];
      const double rr64 = s_sc[1];
      if (bb == 0.0) {
        for (int k = gtid; k < DIM * nh1; k += gstride) a.x[k] = 0.0;
        finish(0, 0, 0.0, 0.0);
        return;
      }
      if (rr64 <= a.tol * a.tol * bb) { finish(inner_total, 0, rr64, bb); return; }
      if (outer >= a.max_outer || inner_total >= a.max_it) { finish(inner_total, 5, rr64, bb); return; }
      // ---- inner FP32 PCG (standard form, exact dot products, three grid barriers
      //      per iteration: in FP32 the scalar recurrence of the FP64 solver
      //      loses too many digits when a step shrinks (r, z) strongly)
      inner_begin();
      float rr = s_f[0], rz = s_f[1], rz_old = rz;
      // relative reduction of this inner solve: inner_tol, or less when a smaller
      // step reaches the FP64 tolerance (0.1 safety factor): a good initial guess
      // then saves inner iterations instead of only whole refinement steps
      const double need = 0.1 * a.tol * sqrt(bb / fmax(rr64, 1e-300));
      const double red_rel = fmax(a.inner_tol, fmin(need, 1.0));
      const float target = (float)(red_rel * red_rel) * rr;
      int it = 0;
      for (;;) {
        if (rr <= target || it >= a.max_inner) break;
        const float beta = it == 0 ? 0.0f : rz / rz_old;
        rz_old = rz;
        // E: FP32 E-vector of M p_new, p_new = invdiag r + beta p, and p_new . M p_new
        // summed element by element inside the sweep
        {
          float pq = 0.0f;
          const bool swept = inner_sweep(beta, pq);
          float acc[1] = {pq};
          block_sum_f(acc);
          if (threadIdx.x == 0) pf[(size_t)2 * G + blockIdx.x] = acc[0];
          if (!swept || !sync()) { finish(inner_total + it, kStatusTimeout, rr64, bb); return; }
        }
        if (threadIdx.x < 32) {
          const float t = warp_sum_partials_f(pf + (size_t)2 * G, G);
          if (threadIdx.x == 0) s_f[2] = rz / t;
        }
        __syncthreads();
        const float alpha = s_f[2];
        {  // one node sweep: q = M p_new gathered, p = p_new, d += alpha p, r -= alpha q,
           // r.r and r.z; one (node, component) per work item, copies through the
           // node-copy table, every load issued first
          float acc[2] = {0, 0};
          if constexpr (P >= 3) {
            // high orders: one node per work item, the loads of all DIM components in
            // flight together (FP32 leaves the registers)
            for (int g = gtid; g < nh1; g += gstride) {
              // copy offsets from the node's coordinates: no table traffic and one
              // memory round trip per node (this sweep is bound by HBM at large sizes)
              int off[1 << DIM];
              node_offsets<DIM, D>(m, g, DIM, off);
              float idg[DIM], pv[DIM], rv[DIM], dv[DIM], ev[DIM][1 << DIM];
#pragma unroll
              for (int c = 0; c < DIM; ++c) {
                const int k = c * nh1 + g;
                idg[c] = __ldg(a.invdiag32 + k);
                pv[c] = a.p32[k];
                rv[c] = a.r32[k];
                dv[c] = a.d32[k];
#pragma unroll
                for (int j = 0; j < (1 << DIM); ++j) ev[c][j] = off[j] >= 0 ? a.evec32[off[j] + c * ND] : 0.0f;
              }
#pragma unroll
              for (int c = 0; c < DIM; ++c) {
                float qv = ev[c][0];
#pragma unroll
                for (int j = 1; j < (1 << DIM); ++j)
                  if (off[j] >= 0) qv += ev[c][j];
                if (idg[c] != 0.0f) {   // constrained DOFs keep p = r = d = 0
                  const int k = c * nh1 + g;
                  const float pn = fmaf(beta, pv[c], idg[c] * rv[c]);
                  const float r2 = fmaf(-alpha, qv, rv[c]);
                  const float z2 = r2 * idg[c];
                  a.p32[k] = pn;
                  a.d32[k] = fmaf(alpha, pn, dv[c]);
                  a.r32[k] = r2;
                  a.z32[k] = z2;
                  acc[0] = fmaf(r2, r2, acc[0]);
                  acc[1] = fmaf(z2, r2, acc[1]);
                }
              }
            }
          } else {
            // low orders: one (node, component) per work item (keeps the register count
            // that allows two CTAs per SM)
            for (int k = gtid; k < DIM * nh1; k += gstride) {
              const int c = DIM == 2 ? (k >= nh1 ? 1 : 0) : (k >= 2 * nh1 ? 2 : (k >= nh1 ? 1 : 0));
              int off[1 << DIM];
              node_table_row<DIM>(a.ncopy, k - c * nh1, off);
              const float idg = __ldg(a.invdiag32 + k);
              const float pv = a.p32[k], rv = a.r32[k], dv = a.d32[k];
              float ev[1 << DIM];
#pragma unroll
              for (int j = 0; j < (1 << DIM); ++j) ev[j] = off[j] >= 0 ? a.evec32[off[j] + c * ND] : 0.0f;
              float qv = ev[0];
#pragma unroll
              for (int j = 1; j < (1 << DIM); ++j)
                if (off[j] >= 0) qv += ev[j];
              if (idg != 0.0f) {   // constrained DOFs keep p = r = d = 0
                const float pn = fmaf(beta, pv, idg * rv);
                const float r2 = fmaf(-alpha, qv, rv);
                const float z2 = r2 * idg;
                a.p32[k] = pn;
                a.d32[k] = fmaf(alpha, pn, dv);
                a.r32[k] = r2;
                a.z32[k] = z2;
                acc[0] = fmaf(r2, r2, acc[0]);
                acc[1] = fmaf(z2, r2, acc[1]);
              }
            }
          }
          block_sum_f(acc);
          if (threadIdx.x == 0) {
            pf[(size_t)0 * G + blockIdx.x] = acc[0];
            pf[(size_t)1 * G + blockIdx.x] = acc[1];
          }
        }
        if (!sync()) { finish(inner_total + it, kStatusTimeout, rr64, bb); return; }
        if (threadIdx.x < 64) {   // r.r on warp 0, r.z on warp 1, side by side
          const int w = threadIdx.x >> 5;
          const float t = warp_sum_partials_f(pf + (size_t)w * G, G);
          if ((threadIdx.x & 31) == 0) s_f[w] = t;
        }
        __syncthreads();
        rr = s_f[0];
        rz = s_f[1];
        ++it;
      }
      inner_total += it;
      // ---- x += d (FP64); every block must see the new x before O-A
      for (int k = gtid; k < DIM * nh1; k += gstride)
        if (a.invdiag[k] != 0.0) a.x[k] += (double)a.d32[k];
      if (!sync()) { finish(inner_total, kStatusTimeout, rr64, bb); return; }
    }
  }

  // ===== setup: geometry at qpoints (J0, detJ0, J0^{-1}, mass data) =======
  // smem: tab | u[CX][ND] | S | g[DIM][CX][NQ] | red
  static constexpr int GE_S = grad_scratch<DIM, D, Q>(CX);
  static constexpr size_t geom_smem() { return sizeof(double) * (TAB + CX * ND + GE_S + DIM * CX * NQ + RED); }
  static __device__ __forceinline__ void body_geom(GeomArgs a) {
    extern __shared__ double sm[];
    double *st = sm, *u = st + TAB, *S = u + CX * ND, *g = S + GE_S, *red = g + DIM * CX * NQ;
    const MeshDesc &m = a.mesh;
    const int e0 = blockIdx.x * NB;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    gather_elem(u, a.x0, DIM, m, e0, nb);
    __syncthreads();
    grad_ref<DIM, D, Q, CX>(u, g, S, st + oB, st + oG);
    double vol = 0.0;
    for (int k = threadIdx.x; k < nb * NQ; k += blockDim.x) {
      const int b = k / NQ, q = k % NQ;
      const size_t e = e0 + b;
      double J[DIM * DIM], Ji[DIM * DIM], det;
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int l = 0; l < DIM; ++l) J[c * DIM + l] = g[(l * CX + b * DIM + c) * NQ + q];
      if constexpr (DIM == 2) {
        det = J[0] * J[3] - J[1] * J[2];
        Ji[0] = J[3] / det; Ji[1] = -J[1] / det; Ji[2] = -J[2] / det; Ji[3] = J[0] / det;
      } else {
        const double c00 = J[4] * J[8] - J[5] * J[7];
        const double c01 = J[5] * J[6] - J[3] * J[8];
        const double c02 = J[3] * J[7] - J[4] * J[6];
        det = J[0] * c00 + J[1] * c01 + J[2] * c02;
        Ji[0] = c00 / det; Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det; Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
        Ji[3] = c01 / det; Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det; Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
        Ji[6] = c02 / det; Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det; Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
      }
      if (!(det > 0.0)) latch_status(a.status, 4);
      double w, iw;
      qweight(st, q, w, iw);
      const double rho0 = a.rho0_in ? a.rho0_in[e * NQ + q] : 1.0;
      a.rho0[e * NQ + q] = rho0;
      a.mq[e * NQ + q] = w * rho0 * det;
#pragma unroll
      for (int r = 0; r < DIM * DIM; ++r) a.jinv0[(e * DIM * DIM + r) * NQ + q] = Ji[r];
      vol = fma(w, det, vol);
    }
    double v1[1] = {vol};
    bsum<1>(v1, red);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = v1[0];
  }

  // ===== setup: per-element diagonal of M (sum_q mq B_i(q)^2) ==============
  static constexpr int DG_S = interp_scratch<DIM, Q, D>(NB);
  static constexpr size_t diag_smem() { return sizeof(double) * (TAB + NB * NQ + DG_S + NB * ND); }
  static __device__ __forceinline__ void body_diag(DiagArgs a) {
    extern __shared__ double sm[];
    double *st = sm, *mq = st + TAB, *S = mq + NB * NQ, *y = S + DG_S;
    const MeshDesc &m = a.mesh;
    const int e0 = blockIdx.x * NB;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    for (int k = threadIdx.x; k < NB * NQ; k += blockDim.x) mq[k] = k / NQ < nb ? a.mq[(size_t)e0 * NQ + k] : 0.0;
    __syncthreads();
    interp<DIM, Q, D, NB>(mq, y, S, st + oB2t);
    for (int k = threadIdx.x; k < nb * ND; k += blockDim.x) a.evec[(size_t)e0 * ND + k] = y[k];
  }

  // ===== setup: element energy-mass inverses (Gauss-Jordan on SPD) ========
  static constexpr size_t emass_smem() { return sizeof(double) * (TAB + NQ + 2 * NL * NL + NL); }
  static __device__ __forceinline__ void body_emass(EmassArgs a) {
    extern __shared__ double sm[];
    double *st = sm, *mq = st + TAB, *A = mq + NQ, *Inv = A + NL * NL, *col = Inv + NL * NL;
    const size_t e = blockIdx.x;
    load_tab(st, a.tab);
    for (int k = threadIdx.x; k < NQ; k += blockDim.x) mq[k] = a.mq[e * NQ + k];
    __syncthreads();
    for (int k = threadIdx.x; k < NL * NL; k += blockDim.x) {   // A_jk = sum_q mq phi_j phi_k
      const int j = k / NL, kk = k % NL;
      double s = 0.0;
      for (int q = 0; q < NQ; ++q) {
        const int qx = q % Q, jx = j % L, kx = kk % L;
        double pj = st[oBl + qx * L + jx], pk = st[oBl + qx * L + kx];
        if constexpr (DIM == 2) {
          const int qy = q / Q, jy = j / L, ky = kk / L;
          pj *= st[oBl + qy * L + jy];
          pk *= st[oBl + qy * L + ky];
        } else {
          const int qy = (q / Q) % Q, jy = (j / L) % L, ky = (kk / L) % L;
          const int qz = q / (Q * Q), jz = j / (L * L), kz = kk / (L * L);
          pj *= st[oBl + qy * L + jy] * st[oBl + qz * L + jz];
          pk *= st[oBl + qy * L + ky] * st[oBl + qz * L + kz];
        }
        s = fma(mq[q] * pj, pk, s);
      }
      A[k] = s;
      Inv[k] = (j == kk) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int piv = 0; piv < NL; ++piv) {
      const double d = A[piv * NL + piv];
      for (int k = threadIdx.x; k < NL; k += blockDim.x) col[k] = A[k * NL + piv];
      __syncthreads();
      for (int k = threadIdx.x; k < NL; k += blockDim.x) {
        A[piv * NL + k] /= d;
        Inv[piv * NL + k] /= d;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < NL * NL; k += blockDim.x) {
        const int i = k / NL, j = k % NL;
        if (i == piv) continue;
        const double f = col[i];
        A[k] = fma(-f, A[piv * NL + j], A[k]);
        Inv[k] = fma(-f, Inv[piv * NL + j], Inv[k]);
      }
      __syncthreads();
    }
    for (int k = threadIdx.x; k < NL * NL; k += blockDim.x) a.me_inv[e * NL * NL + k] = Inv[k];
  }

  // ===== initial energy: element L2 projection of p0/((gamma-1) rho0) =====
  // smem: tab | u[CX][ND] | S | xq[CX][NQ] | sq[NB][NQ] | rhs[NB][NL]
  static constexpr int IE_S = max3(interp_scratch<DIM, D, Q>(CX), interp_scratch<DIM, Q, L>(NB), 0);
  static constexpr size_t init_e_smem() {
    return sizeof(double) * (TAB + CX * ND + IE_S + CX * NQ + NB * NQ + NB * NL);
  }
  static __device__ __forceinline__ void body_init_e(InitEArgs a) {
    extern __shared__ double sm[];
    double *st = sm, *u = st + TAB, *S = u + CX * ND, *xq = S + IE_S, *sq = xq + CX * NQ, *rhs = sq + NB * NQ;
    const MeshDesc &m = a.mesh;
    const int e0 = blockIdx.x * NB;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    gather_elem(u, a.x0, DIM, m, e0, nb);
    __syncthreads();
    interp<DIM, D, Q, CX>(u, xq, S, st + oB);
    const double pi = 3.141592653589793;
    for (int k = threadIdx.x; k < NB * NQ; k += blockDim.x) {
      const int b = k / NQ, q = k % NQ;
      double val = 0.0;
      if (b < nb) {
        const size_t eq = (size_t)(e0 + b) * NQ + q;
        const double X = xq[(b * DIM + 0) * NQ + q], Y = xq[(b * DIM + 1) * NQ + q];
        const double Z = DIM == 3 ? xq[(b * DIM + DIM - 1) * NQ + q] : 0.0;
        const double rho0 = a.rho0[eq];
        double pr;
        if (a.problem == 0) {
          if (DIM == 2) pr = 0.25 * rho0 * (cos(2 * pi * X) + cos(2 * pi * Y)) + 1.0;
          else pr = 100.0 + rho0 / 16.0 * (cos(2 * pi * X) + cos(2 * pi * Y)) * (cos(2 * pi * Z) + 2.0);
        } else {
          const double r = sqrt(X * X + Y * Y);
          if (r < 0.2) pr = 5.0 + 12.5 * r * r;
          else if (r < 0.4) pr = 9.0 - 4.0 * log(0.2) + 12.5 * r * r - 20.0 * r + 4.0 * log(r);
          else pr = 3.0 + 4.0 * log(2.0);
        }
        val = a.mq[eq] * pr / ((a.gamma - 1.0) * rho0);
      }
      sq[k] = val;
    }
    __syncthreads();
    interp<DIM, Q, L, NB>(sq, rhs, S, st + oBlt);
    for (int k = threadIdx.x; k < nb * NL; k += blockDim.x) {
      const int b = k / NL, j = k % NL;
      double s;
      apply_me_inv(a.me_inv, rhs + b * NL, e0 + b, j, s);
      a.e[(size_t)e0 * NL + k] = s;
    }
  }

  // Adjugate A = adj(J) = det(J) J^-1 (row-major, A[l][c]) and det J at qpoint q of
  // element b from reference gradients g[l][b*DIM + c][q] = dx_c/dxi_l (C = CX).
  static __device__ __forceinline__ void adjugate(const double *g, int b, int q, double *A, double &det) {
    double J[DIM * DIM];   // J[c][l] = dx_c/dxi_l
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int l = 0; l < DIM; ++l) J[c * DIM + l] = g[(l * CX + b * DIM + c) * NQ + q];
    if constexpr (DIM == 2) {
      A[0] = J[3]; A[1] = -J[1]; A[2] = -J[2]; A[3] = J[0];
      det = J[0] * J[3] - J[1] * J[2];
    } else {
      A[0] = J[4] * J[8] - J[5] * J[7]; A[1] = J[2] * J[7] - J[1] * J[8]; A[2] = J[1] * J[5] - J[2] * J[4];
      A[3] = J[5] * J[6] - J[3] * J[8]; A[4] = J[0] * J[8] - J[2] * J[6]; A[5] = J[2] * J[3] - J[0] * J[5];
      A[6] = J[3] * J[7] - J[4] * J[6]; A[7] = J[1] * J[6] - J[0] * J[7]; A[8] = J[0] * J[4] - J[1] * J[3];
      det = J[0] * A[0] + J[1] * A[3] + J[2] * A[6];
    }
  }

  // ===== stiffness (diffusion) operator, S_ij = int grad w_i . grad w_j dx ==========
  // (Sections 2.1, 3.3: the hyper-viscosity operator; Section 3.1 decomposition with
  // the reference gradients as B and G below as the qpoint data D.)
  static constexpr int NS = DIM * (DIM + 1) / 2;   // upper triangle of a symmetric d x d
  // Setup on the mesh at node positions x: G = omega adj(J) adj(J)^T / det J
  // (= omega det J J^-1 J^-T) as [NE][NS][NQ] with (l, m >= l) row by row, the
  // unit-density mass data omega det J and the element diagonal of that mass matrix.
  // smem: tab | xu[CX][ND] | S | g[DIM][CX][NQ] | mqs[NB][NQ] | y[NB][ND]
  static constexpr int SS_S = max3(grad_scratch<DIM, D, Q>(CX), interp_scratch<DIM, Q, D>(NB), 0);
  static constexpr size_t stiff_setup_smem() {
    return sizeof(double) * (TAB + CX * ND + SS_S + DIM * CX * NQ + NB * NQ + NB * ND);
  }
  static __device__ __forceinline__ void body_stiff_setup(const StiffArgs &a, int e0) {
    extern __shared__ double sm[];
    double *st = sm, *xu = st + TAB, *S = xu + CX * ND, *g = S + SS_S, *mqs = g + DIM * CX * NQ, *y = mqs + NB * NQ;
    const MeshDesc &m = a.mesh;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    gather_elem(xu, a.x, DIM, m, e0, nb);
    __syncthreads();
    grad_ref<DIM, D, Q, CX>(xu, g, S, st + oB, st + oG);
    for (int k = threadIdx.x; k < NB * NQ; k += blockDim.x) {
      const int b = k / NQ, q = k % NQ;
      double mq = 0.0;
      if (b < nb) {
        double A[DIM * DIM], det, w, iw;
        adjugate(g, b, q, A, det);
        if (!(det > 0.0)) latch_status(a.status, 4);
        qweight(st, q, w, iw);
        mq = w * det;
        const double s = w / det;
        double *Ge = a.G + (size_t)(e0 + b) * NS * NQ + q;
        int r = 0;
#pragma unroll
        for (int l = 0; l < DIM; ++l)
#pragma unroll
          for (int n = l; n < DIM; ++n) {
            double t = 0.0;
#pragma unroll
            for (int c = 0; c < DIM; ++c) t = fma(A[l * DIM + c], A[n * DIM + c], t);
            Ge[(size_t)(r++) * NQ] = s * t;
          }
        a.mq[(size_t)(e0 + b) * NQ + q] = mq;
      }
      mqs[k] = mq;
    }
    __syncthreads();
    interp<DIM, Q, D, NB>(mqs, y, S, st + oB2t);   // sum_q mq B_i(q)^2
    for (int k = threadIdx.x; k < nb * ND; k += blockDim.x) a.dvec[(size_t)e0 * ND + k] = y[k];
  }
  // Action on the DIM components of an H1 field: y_e = sum_q ghat^T G(q) ghat u_e.
  // smem: tab | u[CX][ND] | S | g[DIM][CX][NQ] | gs[NB][NS][NQ]
  static constexpr int SM_S = grad_scratch<DIM, D, Q>(CX);
  static constexpr size_t stiff_smem() {
    return sizeof(double) * (TAB + CX * ND + SM_S + DIM * CX * NQ + NB * NS * NQ);
  }
  static __device__ __forceinline__ void body_stiff(const StiffArgs &a, int e0) {
    extern __shared__ double sm[];
    double *st = sm, *u = st + TAB, *S = u + CX * ND, *g = S + SM_S, *gs = g + DIM * CX * NQ;
    const MeshDesc &m = a.mesh;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    gather_elem(u, a.u, DIM, m, e0, nb);
    for (int k = threadIdx.x; k < NB * NS * NQ; k += blockDim.x)   // one contiguous block per CTA
      gs[k] = k / (NS * NQ) < nb ? a.G[(size_t)e0 * NS * NQ + k] : 0.0;
    __syncthreads();
    grad_ref<DIM, D, Q, CX>(u, g, S, st + oB, st + oG);
    for (int k = threadIdx.x; k < CX * NQ; k += blockDim.x) {
      const int q = k % NQ, bc = k / NQ, b = bc / DIM;
      double gl[DIM], Gs[NS];
#pragma unroll
      for (int l = 0; l < DIM; ++l) gl[l] = g[(l * CX + bc) * NQ + q];
#pragma unroll
      for (int r = 0; r < NS; ++r) Gs[r] = gs[(b * NS + r) * NQ + q];
#pragma unroll
      for (int l = 0; l < DIM; ++l) {
        double t = 0.0;
#pragma unroll
        for (int n = 0; n < DIM; ++n) {
          const int lo = l < n ? l : n, hi = l < n ? n : l;
          t = fma(Gs[lo * DIM - lo * (lo - 1) / 2 + (hi - lo)], gl[n], t);
        }
        g[(l * CX + bc) * NQ + q] = t;
      }
    }
    __syncthreads();
    grad_ref_t<DIM, D, Q, CX>(g, u, S, st + oBt, st + oGt);
    for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x) a.evec[(size_t)e0 * DIM * ND + k] = u[k];
  }

  // ===== mesh optimisation (TMOP, Sections 2.2 and 3.4), fully matrix-free =======
  // Target W = h I (W^-1 = I/h, det W = h^d), T = A W^-1 with A = dx/dxbar; shape
  // metrics mu_2 = |T|^2/(2 det T) - 1 (2D) and mu_303 = |T|^2/(3 det T^(2/3)) - 1 (3D);
  // limiting term lim * |x - x0|^2 (lim = gamma/d^2), both integrated with w_q det W.
  // Every quantity at the qpoints is computed on the fly (no stored qpoint data).
  enum { TM_OBJ = 0, TM_GRAD = 1, TM_HESS = 2, TM_DIAG = 3 };
  static constexpr int NPAIR = NS;   // (n, p >= n) pairs of the diagonal blocks

  // Cofactor C = d(det T)/dT (row-major) and det T.
  static __device__ __forceinline__ double cofactor(const double *T, double *C) {
    if constexpr (DIM == 2) {
      C[0] = T[3]; C[1] = -T[2]; C[2] = -T[1]; C[3] = T[0];
      return T[0] * T[3] - T[1] * T[2];
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) {   // row a of C = row b x row c, (a, b, c) cyclic
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        C[a * 3 + 0] = T[b * 3 + 1] * T[c * 3 + 2] - T[b * 3 + 2] * T[c * 3 + 1];
        C[a * 3 + 1] = T[b * 3 + 2] * T[c * 3 + 0] - T[b * 3 + 0] * T[c * 3 + 2];
        C[a * 3 + 2] = T[b * 3 + 0] * T[c * 3 + 1] - T[b * 3 + 1] * T[c * 3 + 0];
      }
      return T[0] * C[0] + T[1] * C[1] + T[2] * C[2];
    }
  }
  // Scalar factors of the metric and its derivatives at one T:
  //   mu, dmu = cT T + cC C,
  //   d2mu[Z] = cZ Z + cTC ((C:Z) T + (T:Z) C) + cCC (C:Z) C + cdC dC[Z].
  struct MetricCoef {
    double mu, cT, cC, cZ, cTC, cCC, cdC;
  };
  static __device__ __forceinline__ MetricCoef metric(double n2, double tau) {
    MetricCoef k;
    if constexpr (DIM == 2) {
      const double it = 1.0 / tau;
      k.mu = 0.5 * n2 * it - 1.0;
      k.cT = it;
      k.cC = -0.5 * n2 * it * it;
      k.cZ = it;
      k.cTC = -it * it;
      k.cCC = n2 * it * it * it;
      k.cdC = -0.5 * n2 * it * it;
    } else {
      const double rc = rcbrt(tau);          // tau^(-1/3)
      const double r = rc * rc;              // tau^(-2/3)
      const double it = r * rc;              // 1/tau
      k.mu = n2 * r * (1.0 / 3.0) - 1.0;
      k.cT = (2.0 / 3.0) * r;
      k.cC = -(2.0 / 9.0) * n2 * r * it;
      k.cZ = (2.0 / 3.0) * r;
      k.cTC = -(4.0 / 9.0) * r * it;
      k.cCC = (10.0 / 27.0) * n2 * r * it * it;
      k.cdC = -(2.0 / 9.0) * n2 * r * it;
    }
    return k;
  }
  // dC[Z] = d/de cof(T + e Z) at e = 0.
  static __device__ __forceinline__ void dcofactor(const double *T, const double *Z, double *dC) {
    if constexpr (DIM == 2) {
      dC[0] = Z[3]; dC[1] = -Z[2]; dC[2] = -Z[1]; dC[3] = Z[0];
    } else {
#pragma unroll
      for (int a = 0; a < 3; ++a) {   // row a: Z_b x T_c + T_b x Z_c
        const int b = (a + 1) % 3, c = (a + 2) % 3;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
          dC[a * 3 + j] = Z[b * 3 + j1] * T[c * 3 + j2] - Z[b * 3 + j2] * T[c * 3 + j1] +
                          T[b * 3 + j1] * Z[c * 3 + j2] - T[b * 3 + j2] * Z[c * 3 + j1];
        }
      }
    }
  }
  // Per-axis-table contraction from the qpoints to the nodes (Q -> D on every axis,
  // tables [D][Q]): out[c][iz][iy][ix] = sum Mx[ix][qx] My[iy][qy] Mz[iz][qz] in[c][qz][qy][qx].
  template <int C>
  static __device__ __forceinline__ void interp_axes_t(const double *in, double *out, double *S, const double *Mx,
                                                       const double *My, const double *Mz) {
    if constexpr (DIM == 2) {
      contract<C * Q, Q, D, 1>(in, S, Mx);
      __syncthreads();
      contract<C, Q, D, D>(S, out, My);
      __syncthreads();
    } else {
      double *t2 = S + C * Q * Q * D;
      contract<C * Q * Q, Q, D, 1>(in, S, Mx);
      __syncthreads();
      contract<C * Q, Q, D, D>(S, t2, My);
      __syncthreads();
      contract<C, Q, D, D * D>(t2, out, Mz);
      __syncthreads();
    }
  }
  // smem per mode (doubles):
  //   OBJ/GRAD: tab | xu[CX][ND] | du[CX][ND] | S | g[DIM][CX][NQ] | dq[CX][NQ] | red
  //   HESS:     tab | xu | uu | S | g[DIM][CX][NQ] | gu[DIM][CX][NQ] | uq[CX][NQ]
  //   DIAG:     tab | xu | y[CX][ND] | S | g[DIM][CX][NQ] | cq[NPAIR][CX][NQ] | mq[NB][NQ] | G2t | GBt
  static constexpr int TM_S = max3(grad_scratch<DIM, D, Q>(CX), interp_scratch<DIM, D, Q>(CX),
                                   interp_scratch<DIM, Q, D>(CX));
  static constexpr int TQD = ((2 * D * Q) + 1) / 2 * 2;
  static constexpr size_t tmop_smem(int mode) {
    return sizeof(double) *
           (mode == TM_HESS ? TAB + 2 * CX * ND + TM_S + 2 * DIM * CX * NQ + CX * NQ
            : mode == TM_DIAG ? TAB + 2 * CX * ND + TM_S + DIM * CX * NQ + NPAIR * CX * NQ + NB * NQ + TQD
                              : TAB + 2 * CX * ND + TM_S + DIM * CX * NQ + CX * NQ + RED);
  }
  template <int MODE>
  static __device__ __forceinline__ void body_tmop(const TmopArgs &a, int e0) {
    extern __shared__ double sm[];
    double *st = sm, *xu = st + TAB, *uu = xu + CX * ND, *S = uu + CX * ND, *g = S + TM_S;
    double *q1 = g + DIM * CX * NQ;   // OBJ/GRAD: dq; HESS: gu; DIAG: cq
    const MeshDesc &m = a.mesh;
    const int nb = min(NB, m.ne - e0);
    const bool lim = a.lim != 0.0 && (MODE == TM_HESS || MODE == TM_DIAG || a.x0 != nullptr);
    load_tab(st, a.tab);
    for (int k = threadIdx.x; k < CX * ND; k += blockDim.x) {
      const int i = k % ND, bc = k / ND, c = bc % DIM, b = bc / DIM;
      double x = 0.0, w = 0.0;
      if (b < nb) {
        const size_t gi = (size_t)c * m.nh1 + h1_node<DIM, D>(m, e0 + b, i);
        x = a.x[gi];
        if (MODE == TM_HESS) w = a.u[gi];
        else if ((MODE == TM_OBJ || MODE == TM_GRAD) && lim) w = x - a.x0[gi];
      }
      xu[k] = x;
      if (MODE != TM_DIAG) uu[k] = w;
    }
    __syncthreads();
    grad_ref<DIM, D, Q, CX>(xu, g, S, st + oB, st + oG);   // A = dx/dxbar
    if (MODE == TM_HESS) {
      grad_ref<DIM, D, Q, CX>(uu, q1, S, st + oB, st + oG);   // du/dxbar
      if (lim) interp<DIM, D, Q, CX>(uu, q1 + DIM * CX * NQ, S, st + oB);
    } else if (MODE != TM_DIAG && lim) {
      interp<DIM, D, Q, CX>(uu, q1, S, st + oB);   // x - x0 at the qpoints
    }
    const double hi = a.h_inv, wdet = a.detW;
    double acc = 0.0;
    for (int k = threadIdx.x; k < NB * NQ; k += blockDim.x) {
      const int b = k / NQ, q = k % NQ;
      if (b >= nb) {
        if (MODE == TM_DIAG)
          for (int r = 0; r < NPAIR * DIM; ++r) q1[(r / DIM * CX + b * DIM + r % DIM) * NQ + q] = 0.0;
        if (MODE == TM_DIAG) q1[NPAIR * CX * NQ + k] = 0.0;
        continue;
      }
      double Tm[DIM * DIM], C[DIM * DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int l = 0; l < DIM; ++l) Tm[c * DIM + l] = hi * g[(l * CX + b * DIM + c) * NQ + q];
      const double tau = cofactor(Tm, C);
      if (!(tau > 0.0)) latch_status(a.status, 4);
      double n2 = 0.0;
#pragma unroll
      for (int r = 0; r < DIM * DIM; ++r) n2 = fma(Tm[r], Tm[r], n2);
      const MetricCoef mc = metric(n2, tau);
      double w, iw;
      qweight(st, q, w, iw);
      const double wq = w * wdet;
      if (MODE == TM_OBJ) {
        double s = mc.mu;
        if (lim) {
          double d2 = 0.0;
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            const double dv = q1[(b * DIM + c) * NQ + q];
            d2 = fma(dv, dv, d2);
          }
          s = fma(a.lim, d2, s);
        }
        acc = fma(wq, s, acc);
      } else if (MODE == TM_GRAD) {
        const double f = wq * hi;   // f[n][a] = w detW / h * dmu_an
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
          for (int n = 0; n < DIM; ++n)
            g[(n * CX + b * DIM + c) * NQ + q] = f * fma(mc.cT, Tm[c * DIM + n], mc.cC * C[c * DIM + n]);
        if (lim)
#pragma unroll
          for (int c = 0; c < DIM; ++c) q1[(b * DIM + c) * NQ + q] *= 2.0 * a.lim * wq;
      } else if (MODE == TM_HESS) {
        double Z[DIM * DIM], dC[DIM * DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
          for (int l = 0; l < DIM; ++l) Z[c * DIM + l] = hi * q1[(l * CX + b * DIM + c) * NQ + q];
        dcofactor(Tm, Z, dC);
        double cz = 0.0, tz = 0.0;
#pragma unroll
        for (int r = 0; r < DIM * DIM; ++r) {
          cz = fma(C[r], Z[r], cz);
          tz = fma(Tm[r], Z[r], tz);
        }
        const double f = wq * hi;
        const double kT = mc.cTC * cz, kC = fma(mc.cTC, tz, mc.cCC * cz);
#pragma unroll
        for (int c = 0; c < DIM; ++c)
#pragma unroll
          for (int n = 0; n < DIM; ++n) {
            const int r = c * DIM + n;
            const double v = fma(mc.cZ, Z[r], fma(kT, Tm[r], fma(kC, C[r], mc.cdC * dC[r])));
            g[(n * CX + b * DIM + c) * NQ + q] = f * v;
          }
        if (lim)
#pragma unroll
          for (int c = 0; c < DIM; ++c) q1[DIM * CX * NQ + (b * DIM + c) * NQ + q] *= 2.0 * a.lim * wq;
      } else {   // TM_DIAG: H_a[n][p] = cZ d_np + cTC (C_ap T_an + T_ap C_an) + cCC C_an C_ap
        const double f = wq * hi * hi;
        int r = 0;
#pragma unroll
        for (int n = 0; n < DIM; ++n)
#pragma unroll
          for (int p = n; p < DIM; ++p, ++r) {
            const double sym = n == p ? 1.0 : 2.0;
#pragma unroll
            for (int c = 0; c < DIM; ++c) {
              const double Can = C[c * DIM + n], Cap = C[c * DIM + p];
              const double Tan = Tm[c * DIM + n], Tap = Tm[c * DIM + p];
              double hv = mc.cTC * fma(Cap, Tan, Tap * Can) + mc.cCC * Can * Cap;
              if (n == p) hv += mc.cZ;
              q1[(r * CX + b * DIM + c) * NQ + q] = sym * f * hv;
            }
          }
        q1[NPAIR * CX * NQ + k] = lim ? 2.0 * a.lim * wq : 0.0;
      }
    }
    if (MODE == TM_OBJ) {
      double v1[1] = {acc};
      bsum<1>(v1, q1 + CX * NQ);
      __shared__ int s_last;
      if (threadIdx.x == 0) {
        a.partials[blockIdx.x] = v1[0];
        __threadfence();
        s_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
      }
      __syncthreads();
      if (!s_last || threadIdx.x >= 32) return;
      __threadfence();
      double sacc = 0.0;
      for (int i = threadIdx.x; i < (int)gridDim.x; i += 32) sacc += ((volatile double *)a.partials)[i];
      sacc = warp_sum(sacc);
      if (threadIdx.x == 0) {
        *a.counter = 0u;
        *a.out = sacc;
      }
      return;
    }
    __syncthreads();
    if (MODE == TM_GRAD || MODE == TM_HESS) {
      grad_ref_t<DIM, D, Q, CX>(g, xu, S, st + oBt, st + oGt);   // sum_q sum_n dw_i/dxbar_n f[n][c]
      const double *lq = MODE == TM_HESS ? q1 + DIM * CX * NQ : q1;
      if (lim) interp<DIM, Q, D, CX>(lq, uu, S, st + oBt);        // sum_q w_i (limiting factor)
      for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x)
        a.evec[(size_t)e0 * DIM * ND + k] = lim ? xu[k] + uu[k] : xu[k];
      return;
    }
    // TM_DIAG: sum over pairs of per-axis contractions with the tables G^2, G B, B^2
    double *G2t = q1 + NPAIR * CX * NQ + NB * NQ, *GBt = G2t + D * Q;
    for (int k = threadIdx.x; k < D * Q; k += blockDim.x) {
      const double gt = st[oGt + k], bt = st[oBt + k];
      G2t[k] = gt * gt;
      GBt[k] = gt * bt;
    }
    __syncthreads();
    double *y = uu;
    for (int k = threadIdx.x; k < CX * ND; k += blockDim.x) xu[k] = 0.0;
    int r = 0;
    for (int n = 0; n < DIM; ++n)
      for (int p = n; p < DIM; ++p, ++r) {
        const double *M[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
          M[ax] = (ax == n && ax == p) ? G2t : (ax == n || ax == p) ? GBt : st + oB2t;
        interp_axes_t<CX>(q1 + r * CX * NQ, y, S, M[0], M[1], M[2]);
        for (int k = threadIdx.x; k < CX * ND; k += blockDim.x) xu[k] += y[k];
        __syncthreads();
      }
    if (lim) {
      interp<DIM, Q, D, NB>(q1 + NPAIR * CX * NQ, y, S, st + oB2t);   // 2 lim w detW w_i^2
      for (int k = threadIdx.x; k < CX * ND; k += blockDim.x) xu[k] += y[(k / (DIM * ND)) * ND + k % ND];
      __syncthreads();
    }
    for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x) a.evec[(size_t)e0 * DIM * ND + k] = xu[k];
  }

  // ----- partially assembled Hessian (a B300 variant of Eq. 7 for repeated products) -----
  // setup: per qpoint the symmetric 2nd-derivative tensor of mu, scaled by w det W / h^2,
  // as the upper triangle of the (a n) x (b p) matrix: [NE][NH2][NQ];
  // apply: y_e = sum_q ghat^T (H : ghat u) + the limiting term, from that data.
  static constexpr int NR = DIM * DIM;
  static constexpr int NH2 = NR * (NR + 1) / 2;
  static __device__ __forceinline__ int hidx(int r, int s) { return r * NR - r * (r - 1) / 2 + (s - r); }
  // d C_an / d T_bp (the cofactor's derivative; C_an does not depend on row a of T)
  static __device__ __forceinline__ double dcof(const double *T, int a, int n, int b, int p) {
    if constexpr (DIM == 2) {
      return (b == 1 - a && p == 1 - n) ? (a == n ? 1.0 : -1.0) : 0.0;
    } else {
      if (a == b || n == p) return 0.0;
      const int c = 3 - a - b, q = 3 - n - p;
      const double s1 = (b - a + 3) % 3 == 1 ? 1.0 : -1.0, s2 = (p - n + 3) % 3 == 1 ? 1.0 : -1.0;
      return s1 * s2 * T[c * 3 + q];
    }
  }
  static __device__ __forceinline__ void body_tmop_pa_setup(const TmopArgs &a, int e0) {
    extern __shared__ double sm[];
    double *st = sm, *xu = st + TAB, *S = xu + 2 * CX * ND, *g = S + TM_S;
    const MeshDesc &m = a.mesh;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    gather_elem(xu, a.x, DIM, m, e0, nb);
    __syncthreads();
    grad_ref<DIM, D, Q, CX>(xu, g, S, st + oB, st + oG);
    const double hi = a.h_inv;
    for (int k = threadIdx.x; k < nb * NQ; k += blockDim.x) {
      const int b = k / NQ, q = k % NQ;
      double Tm[NR], C[NR];
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int l = 0; l < DIM; ++l) Tm[c * DIM + l] = hi * g[(l * CX + b * DIM + c) * NQ + q];
      const double tau = cofactor(Tm, C);
      if (!(tau > 0.0)) latch_status(a.status, 4);
      double n2 = 0.0;
#pragma unroll
      for (int r = 0; r < NR; ++r) n2 = fma(Tm[r], Tm[r], n2);
      const MetricCoef mc = metric(n2, tau);
      double w, iw;
      qweight(st, q, w, iw);
      const double f = w * a.detW * hi * hi;
      double *He = a.pa + (size_t)(e0 + b) * NH2 * NQ + q;
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int s = r; s < NR; ++s) {
          const int ai = r / DIM, ni = r % DIM, bi = s / DIM, pi = s % DIM;
          double h = mc.cTC * fma(Tm[r], C[s], Tm[s] * C[r]) + mc.cCC * C[r] * C[s] + mc.cdC * dcof(Tm, ai, ni, bi, pi);
          if (r == s) h += mc.cZ;
          He[(size_t)hidx(r, s) * NQ] = f * h;
        }
    }
  }
  static __device__ __forceinline__ void body_tmop_pa_apply(const TmopArgs &a, int e0) {
    extern __shared__ double sm[];
    double *st = sm, *uu = st + TAB, *yv = uu + CX * ND, *S = yv + CX * ND, *g = S + TM_S;
    double *uq = g + DIM * CX * NQ;
    const MeshDesc &m = a.mesh;
    const int nb = min(NB, m.ne - e0);
    const bool lim = a.lim != 0.0;
    load_tab(st, a.tab);
    gather_elem(uu, a.u, DIM, m, e0, nb);
    __syncthreads();
    grad_ref<DIM, D, Q, CX>(uu, g, S, st + oB, st + oG);
    if (lim) interp<DIM, D, Q, CX>(uu, uq, S, st + oB);
    for (int k = threadIdx.x; k < nb * NQ; k += blockDim.x) {
      const int b = k / NQ, q = k % NQ;
      double Z[NR];
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int l = 0; l < DIM; ++l) Z[c * DIM + l] = g[(l * CX + b * DIM + c) * NQ + q];
      const double *He = a.pa + (size_t)(e0 + b) * NH2 * NQ + q;
      double y[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) y[r] = 0.0;
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int s = r; s < NR; ++s) {
          const double h = He[(size_t)hidx(r, s) * NQ];
          y[r] = fma(h, Z[s], y[r]);
          if (s != r) y[s] = fma(h, Z[r], y[s]);
        }
#pragma unroll
      for (int c = 0; c < DIM; ++c)
#pragma unroll
        for (int n = 0; n < DIM; ++n) g[(n * CX + b * DIM + c) * NQ + q] = y[c * DIM + n];
      if (lim) {
        double w, iw;
        qweight(st, q, w, iw);
#pragma unroll
        for (int c = 0; c < DIM; ++c) uq[(b * DIM + c) * NQ + q] *= 2.0 * a.lim * w * a.detW;
      }
    }
    __syncthreads();
    grad_ref_t<DIM, D, Q, CX>(g, yv, S, st + oBt, st + oGt);
    if (lim) interp<DIM, Q, D, CX>(uq, uu, S, st + oBt);
    for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x)
      a.evec[(size_t)e0 * DIM * ND + k] = lim ? yv[k] + uu[k] : yv[k];
  }

  // ===== remap phase (Section 3.5): one stage on the mesh x(tau) = x0 + tau u ====
  // Per element and qpoint of x(tau): mq = omega detJ (the mass data of M(tau)) and
  // the advection data adv_l = omega detJ (J^-1 u)_l = omega (adj(J) u)_l, kept in
  // shared memory only. From them, in the same pass: the element diagonal of M(tau)
  // (sum_q mq B_i(q)^2) and the element contributions of K(tau) w,
  //     (K w)_i = sum_q B_i(q) sum_l adv_l(q) dw/dxi_l(q),   w = v + s k.
  // smem: tab | xu[CX][ND] | uu[CX][ND] | vv[CX][ND] | S | g[DIM][CX][NQ] |
  //       uq[CX][NQ] | adv[DIM][NB][NQ] | mqs[NB][NQ]
  static constexpr int RM_S = max3(grad_scratch<DIM, D, Q>(CX), interp_scratch<DIM, D, Q>(CX),
                                   interp_scratch<DIM, Q, D>(CX));
  static constexpr size_t remap_smem() {
    return sizeof(double) * (TAB + 3 * CX * ND + RM_S + DIM * CX * NQ + CX * NQ + DIM * NB * NQ + NB * NQ);
  }
  static __device__ __forceinline__ void body_remap(const RemapArgs &a, int e0) {
    extern __shared__ double sm[];
    double *st = sm, *xu = st + TAB, *uu = xu + CX * ND, *vv = uu + CX * ND, *S = vv + CX * ND;
    double *g = S + RM_S, *uq = g + DIM * CX * NQ, *adv = uq + CX * NQ, *mqs = adv + DIM * NB * NQ;
    const MeshDesc &m = a.mesh;
    const int nb = min(NB, m.ne - e0);
    load_tab(st, a.tab);
    for (int k = threadIdx.x; k < CX * ND; k += blockDim.x) {
      const int i = k % ND, bc = k / ND, c = bc % DIM, b = bc / DIM;
      double x = 0.0, u = 0.0, w = 0.0;
      if (b < nb) {
        const size_t gi = (size_t)c * m.nh1 + h1_node<DIM, D>(m, e0 + b, i);
        u = a.u[gi];
        x = fma(a.tau, u, a.x0[gi]);
        if (a.evec) w = a.k ? fma(a.s, a.k[gi], a.v[gi]) : a.v[gi];
      }
      xu[k] = x;
      uu[k] = u;
      vv[k] = w;
    }
    __syncthreads();
    grad_ref<DIM, D, Q, CX>(xu, g, S, st + oB, st + oG);   // J(tau) = dx/dxi
    interp<DIM, D, Q, CX>(uu, uq, S, st + oB);             // u at the qpoints
    for (int k = threadIdx.x; k < NB * NQ; k += blockDim.x) {
      const int b = k / NQ, q = k % NQ;
      double mq = 0.0, al[DIM];
#pragma unroll
      for (int l = 0; l < DIM; ++l) al[l] = 0.0;
      if (b < nb) {
        double A[DIM * DIM], det;
        adjugate(g, b, q, A, det);
        if (!(det > 0.0)) latch_status(a.status, 4);
        double w, iw;
        qweight(st, q, w, iw);
        mq = w * det;
        a.mq[(size_t)(e0 + b) * NQ + q] = mq;
#pragma unroll
        for (int l = 0; l < DIM; ++l) {
          double s = 0.0;
#pragma unroll
          for (int c = 0; c < DIM; ++c) s = fma(A[l * DIM + c], uq[(b * DIM + c) * NQ + q], s);
          al[l] = w * s;
        }
      }
      mqs[k] = mq;
#pragma unroll
      for (int l = 0; l < DIM; ++l) adv[l * NB * NQ + k] = al[l];
    }
    __syncthreads();
    if (a.dvec) {
      interp<DIM, Q, D, NB>(mqs, xu, S, st + oB2t);   // sum_q mq B_i(q)^2
      for (int k = threadIdx.x; k < nb * ND; k += blockDim.x) a.dvec[(size_t)e0 * ND + k] = xu[k];
    }
    if (!a.evec) return;
    grad_ref<DIM, D, Q, CX>(vv, g, S, st + oB, st + oG);   // dw/dxi
    for (int k = threadIdx.x; k < CX * NQ; k += blockDim.x) {
      const int q = k % NQ, bc = k / NQ, b = bc / DIM;
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < DIM; ++l) s = fma(adv[(l * NB + b) * NQ + q], g[(l * CX + bc) * NQ + q], s);
      uq[k] = s;
    }
    __syncthreads();
    interp<DIM, Q, D, CX>(uq, uu, S, st + oBt);   // B^T
    for (int k = threadIdx.x; k < nb * DIM * ND; k += blockDim.x) a.evec[(size_t)e0 * DIM * ND + k] = uu[k];
  }
};

// Kernel entry points (free templates; the bodies live in Family).
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_qdata(QdataArgs a) { Family<DIM, P, Q>::body_qdata(a, blockIdx.x * Family<DIM, P, Q>::NB); }
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_force(ForceArgs a) { Family<DIM, P, Q>::body_force(a, blockIdx.x * Family<DIM, P, Q>::NB); }
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_force_t(ForceTArgs a) { Family<DIM, P, Q>::body_force_t(a, blockIdx.x * Family<DIM, P, Q>::NB); }
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_mass(MassArgs a) { Family<DIM, P, Q>::body_mass(a, blockIdx.x * Family<DIM, P, Q>::NB); }
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::TC, Family<DIM, P, Q>::CG_MINB) k_cg(CgArgs a) {
  Family<DIM, P, Q>::body_cg(a);
}
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::TC, Family<DIM, P, Q>::CGIR_MINB) k_cg_ir(CgIrArgs a) {
  Family<DIM, P, Q>::body_cg_ir(a);
}
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_geom(GeomArgs a) { Family<DIM, P, Q>::body_geom(a); }
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_diag(DiagArgs a) { Family<DIM, P, Q>::body_diag(a); }
template <int DIM, int P, int Q>
__global__ void k_emass(EmassArgs a) { Family<DIM, P, Q>::body_emass(a); }
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_init_e(InitEArgs a) { Family<DIM, P, Q>::body_init_e(a); }
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_remap(RemapArgs a) { Family<DIM, P, Q>::body_remap(a, blockIdx.x * Family<DIM, P, Q>::NB); }
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_stiff_setup(StiffArgs a) { Family<DIM, P, Q>::body_stiff_setup(a, blockIdx.x * Family<DIM, P, Q>::NB); }
template <int DIM, int P, int Q>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_stiff(StiffArgs a) { Family<DIM, P, Q>::body_stiff(a, blockIdx.x * Family<DIM, P, Q>::NB); }
template <int DIM, int P, int Q, int MODE>
__global__ void __launch_bounds__(Family<DIM, P, Q>::THREADS) k_tmop(TmopArgs a) {
  if constexpr (MODE == 4) Family<DIM, P, Q>::body_tmop_pa_setup(a, blockIdx.x * Family<DIM, P, Q>::NB);
  else if constexpr (MODE == 5) Family<DIM, P, Q>::body_tmop_pa_apply(a, blockIdx.x * Family<DIM, P, Q>::NB);
  else Family<DIM, P, Q>::template body_tmop<MODE>(a, blockIdx.x * Family<DIM, P, Q>::NB);
}

}  // namespace lh

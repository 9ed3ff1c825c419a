// Per-wavevector depth operators of the discretised Mindlin and Boussinesq operators.
//
// For one in-plane mode q = 2 pi (k1/L1, k2/L2) the Mindlin displacement gradient at the
// depth node x3^i is (Eq. 2gradient, Eq. jump, Eq. mindlin_B_U, Thm 1)
//   grad N[w](q, x3^i) = - int grad^2 U_inf(-q, y3 - x3^i) : w_h(q, y3) dy3
//                        - ([[grad U_inf]] : w(q, x3^i)) x e3  +  image term,
// with w_h the piecewise-linear interpolant of the nodal coefficients (Sec. 3.2).
//
// GB300 formulation (the paper's element integrals, evaluated exactly, reorganised):
// * Frame: the tensors are rotated so that q lies along x1; with Delta(-q) = (-i, 0, 0)
//   every kernel coefficient of Table 1 becomes a constant and the contraction of the
//   4th-order kernels with w collapses to five rotated components of w plus one scalar
//   (Delta^+-.w.Delta^+-) per branch; the in-plane component perpendicular to q has no
//   strain (eps_pp = 0).
// * Depth integral: the g0/g1 kernels are exponentials exp(-q|y3 - x3|) times
//   polynomials, so the integrals over all elements above (g^- branch) and below (g^+
//   branch) of node i follow from those of node i-1 / i+1 by the exact one-element
//   recursions  M0 <- e^{-qh} M0 + element,  M1 <- e^{-qh}(M1 -+ qh M0) + element,
//   with the linear-element integrals of Eq. (int_g0)/(int_g1) in closed form.  This
//   replaces the cutoff of Sec. 3.2 (no approximation) and costs O(Nz) per mode.
// * Parallelism: a CTA holds KT consecutive k1 columns (one k2) for all depth nodes in
//   shared memory; the depth range is cut into chunks of C nodes, one thread per
//   (chunk, k1).  Each chunk first computes its local contribution (from zero), the
//   carries of the two recursions are folded across chunks in shared memory, then every
//   chunk re-runs its recursion from the exact carries and writes its nodes.
// * Image term: the surface traction of the full-space field needs the + branch at
//   x3 = 0, i.e. the fully folded carry; the cancelling Boussinesq field is then a
//   closed form exp(-q z)(P + q z Q) in the rotated frame.
// * q = 0 (mode k = 0): laminate solution (sigma_i3 = 0, eps_ab = 0).  k2 = N2/2
//   (not in Z^2_N): no operator term, so sigma_hat = -w_hat (stress) or 0 (strain).
#include <string.h>

#include <algorithm>

#include "fvim_internal.cuh"

namespace {

constexpr int KT_MAX = 16;  // k1 columns per CTA (128-byte rows in FP32)
constexpr double kTwoPi = 6.283185307179586476925;

template <typename T> __device__ __forceinline__ T dexp(T x);
template <> __device__ __forceinline__ float dexp<float>(float x) { return expf(x); }
template <> __device__ __forceinline__ double dexp<double>(double x) { return exp(x); }

// wait for phase 0 of the mbarrier at shared address bar, at most limit_ns nanoseconds of the
// global timer and at most 2^24 polls (should the timer not advance); true when the phase
// completed
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned long long limit_ns) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (int it = 0; it < (1 << 24); ++it) {
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(bar)
                 : "memory");
    if (ok) return true;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) return false;
  }
  return false;
}

// Linear-element integrals of Eq. (int_g0)/(int_g1): with a = q h,
//   I_n(a) = int_0^1 s^n exp(-a s) ds,  n = 0, 1, 2,
// closed form for a above a threshold, Taylor series below it (no cancellation).
template <typename T> struct Elem {
  T E, a, h, hI0mI1, hI1, ahI1mI2, ahI2;
};

template <typename T> __device__ __forceinline__ Elem<T> elem_coef(T q, T h) {
  Elem<T> c;
  const T a = q * h;
  const T E = dexp<T>(-a);
  T I0, I1, I2;
  const T thr = sizeof(T) == 4 ? (T)1.0 : (T)0.5;
  if (a < thr) {
    // I_n(a) = sum_m (-a)^m / (m! (n + m + 1)); the reciprocals are compile-time constants
    constexpr int M = sizeof(T) == 4 ? 12 : 18;
    T term = 1, s0 = 0, s1 = 0, s2 = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      s0 += term * (T)(1.0 / (m + 1));
      s1 += term * (T)(1.0 / (m + 2));
      s2 += term * (T)(1.0 / (m + 3));
      term *= -a * (T)(1.0 / (m + 1));
    }
    I0 = s0; I1 = s1; I2 = s2;
  } else {
    const T ia = (T)1 / a;
    I0 = ((T)1 - E) * ia;
    I1 = ((T)1 - E * ((T)1 + a)) * ia * ia;
    I2 = ((T)2 - E * (a * a + (T)2 * a + (T)2)) * ia * ia * ia;
  }
  c.E = E;
  c.a = a;
  c.h = h;
  c.hI0mI1 = h * (I0 - I1);
  c.hI1 = h * I1;
  c.ahI1mI2 = a * h * (I1 - I2);
  c.ahI2 = a * h * I2;
  return c;
}

// moments of one branch: m = int g0 w_h for the rotated components
// (qq, 33, p3, q3, qp); n = int g1 (D.w_h.D) with D = Delta^{+-}(-q) in the rotated frame
template <typename V> struct Mom {
  V m[5];
  V n;
};

// rotated storage order: 0 qq, 1 pp, 2 33, 3 p3, 4 q3, 5 qp; moment j -> rotated j ? j + 1 : 0

template <typename V> __device__ __forceinline__ void mom_zero(Mom<V>& M) {
#pragma unroll
  for (int j = 0; j < 5; ++j) M.m[j] = mk<V>(0, 0);
  M.n = mk<V>(0, 0);
}

// scalar Delta^-.X.Delta^- (A branch, sgn = -1) or Delta^+.X.Delta^+ (P branch, sgn = +1)
// for the rotated components qq, 33, q3:  -X_qq + X_33 + sgn 2i X_q3
template <typename V> __device__ __forceinline__ V nscal(V qq, V z33, V q3, int sgn) {
  const V r = csub(z33, qq);
  return caxpy_i(r, sgn > 0 ? (decltype(V::x))2 : (decltype(V::x))-2, q3);
}

// forward step of the g^- moments from node i to node i+1 over element [i, i+1]
template <typename T, typename V>
__device__ __forceinline__ void stepA(Mom<V>& A, const Elem<T>& c, const V* wi, const V* wj) {
  const V n_old = nscal(A.m[0], A.m[1], A.m[3], -1);
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int r = (j == 0) ? 0 : j + 1;
    V v = cscale(A.m[j], c.E);
    v = caxpy(v, c.hI1, wi[r]);
    v = caxpy(v, c.hI0mI1, wj[r]);
    A.m[j] = v;
  }
  const V ni = nscal(wi[0], wi[2], wi[4], -1);
  const V nj = nscal(wj[0], wj[2], wj[4], -1);
  V v = cscale(caxpy(A.n, -c.a, n_old), c.E);
  v = caxpy(v, -c.ahI2, ni);
  v = caxpy(v, -c.ahI1mI2, nj);
  A.n = v;
}

// backward step of the g^+ moments from node i+1 to node i over element [i, i+1]
template <typename T, typename V>
__device__ __forceinline__ void stepP(Mom<V>& P, const Elem<T>& c, const V* wi, const V* wj) {
  const V n_old = nscal(P.m[0], P.m[1], P.m[3], +1);
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int r = (j == 0) ? 0 : j + 1;
    V v = cscale(P.m[j], c.E);
    v = caxpy(v, c.hI0mI1, wi[r]);
    v = caxpy(v, c.hI1, wj[r]);
    P.m[j] = v;
  }
  const V ni = nscal(wi[0], wi[2], wi[4], +1);
  const V nj = nscal(wj[0], wj[2], wj[4], +1);
  V v = cscale(caxpy(P.n, c.a, n_old), c.E);
  v = caxpy(v, c.ahI1mI2, ni);
  v = caxpy(v, c.ahI2, nj);
  P.n = v;
}

// propagate a branch across a depth span with a = q * span (no source inside)
template <typename T, typename V>
__device__ __forceinline__ void propA(Mom<V>& A, T a) {
  const T E = dexp<T>(-a);
  const V n0 = nscal(A.m[0], A.m[1], A.m[3], -1);
  A.n = cscale(caxpy(A.n, -a, n0), E);
#pragma unroll
  for (int j = 0; j < 5; ++j) A.m[j] = cscale(A.m[j], E);
}
// with E = e^{-a} given
template <typename T, typename V>
__device__ __forceinline__ void propP_E(Mom<V>& P, T a, T E) {
  const V n0 = nscal(P.m[0], P.m[1], P.m[3], +1);
  P.n = cscale(caxpy(P.n, a, n0), E);
#pragma unroll
  for (int j = 0; j < 5; ++j) P.m[j] = cscale(P.m[j], E);
}
template <typename T, typename V>
__device__ __forceinline__ void propP(Mom<V>& P, T a) {
  propP_E(P, a, dexp<T>(-a));
}
template <typename V> __device__ __forceinline__ void mom_add(Mom<V>& a, const Mom<V>& b) {
#pragma unroll
  for (int j = 0; j < 5; ++j) a.m[j] = cadd(a.m[j], b.m[j]);
  a.n = cadd(a.n, b.n);
}

// Kelvin part of the strain (full-space field, Eq. 2gradient + Eq. jump) in the rotated
// frame from the two branch moments and the nodal eigenstress w (rotated, 6 comps).
template <typename T, typename V>
__device__ __forceinline__ void kelvin_strain(const Mom<V>& A, const Mom<V>& P, const V* w, T q, T nu, T mu,
                                              V* e) {
  const T K = (T)1 / ((T)8 * mu * (nu - (T)1));
  const V S0 = cadd(A.m[0], P.m[0]), S2 = cadd(A.m[1], P.m[1]), S3 = cadd(A.m[2], P.m[2]);
  const V S4 = cadd(A.m[3], P.m[3]), S5 = cadd(A.m[4], P.m[4]);
  const V D0 = csub(A.m[0], P.m[0]), D2 = csub(A.m[1], P.m[1]), D3 = csub(A.m[2], P.m[2]);
  const V D4 = csub(A.m[3], P.m[3]), D5 = csub(A.m[4], P.m[4]);
  const V An = A.n, Pn = P.n;
  // eps_qq = q K [(4nu-3) S0 + S2 + 4i(nu-1) D4 + An - Pn]
  V t = cscale(S0, (T)4 * nu - (T)3);
  t = cadd(t, S2);
  t = caxpy_i(t, (T)4 * (nu - (T)1), D4);
  t = cadd(t, csub(An, Pn));
  e[0] = cscale(t, q * K);
  e[1] = mk<V>(0, 0);
  // eps_33 = K [q (S0 - (4nu-1) S2 + 4i nu D4 - An + Pn) + 4(2nu-1) w33]
  t = caxpy(S0, -((T)4 * nu - (T)1), S2);
  t = caxpy_i(t, (T)4 * nu, D4);
  t = cadd(t, csub(Pn, An));
  t = cscale(t, q);
  t = caxpy(t, (T)4 * ((T)2 * nu - (T)1), w[2]);
  e[2] = cscale(t, K);
  // eps_p3 = (q(-S3 + i D5) + 2 w_p3) / (4 mu)
  t = caxpy_i(cscale(S3, (T)-1), (T)1, D5);
  t = cscale(t, q);
  t = caxpy(t, (T)2, w[3]);
  e[3] = cscale(t, (T)1 / ((T)4 * mu));
  // eps_q3 = K [q(i(2(nu-1) D0 + 2 nu D2 + An + Pn) + 2 S4) + 4(nu-1) w_q3]
  V u = cscale(D0, (T)2 * (nu - (T)1));
  u = caxpy(u, (T)2 * nu, D2);
  u = cadd(u, cadd(An, Pn));
  t = caxpy_i(cscale(S4, (T)2), (T)1, u);
  t = cscale(t, q);
  t = caxpy(t, (T)4 * (nu - (T)1), w[4]);
  e[4] = cscale(t, K);
  // eps_qp = q (i D3 + S5) / (4 mu)
  t = caxpy_i(S5, (T)1, D3);
  e[5] = cscale(t, q / ((T)4 * mu));
}

// strain of the Boussinesq-Cerruti field of a surface traction t (rotated frame, force on
// the body per unit area, Eq. B:fourier with its gradient recurrence) at zeta = q z
template <typename T, typename V>
__device__ __forceinline__ void bous_strain_add(const V* tr, T zeta, T ex, T nu, T imu, V* e) {
  // ex = exp(-zeta), imu = 1 / mu
  const T c1 = ex * imu, c2 = (T)0.5 * ex * imu;
  const V t0 = tr[0], t1 = tr[1], t2 = tr[2];
  // qq: ((1-nu) i t0 + (nu - 1/2) t2 + zeta(-i t0/2 + t2/2)) / mu
  //   = ((1 - nu) - zeta/2) i t0 + ((nu - 1/2) + zeta/2) t2
  V v = caxpy_i(cscale(t2, nu - (T)0.5 + (T)0.5 * zeta), (T)1 - nu - (T)0.5 * zeta, t0);
  e[0] = caxpy(e[0], c1, v);
  // 33: (-2 i nu t0 + (2nu-1) t2 + zeta (i t0 - t2)) / (2 mu)
  //   = (zeta - 2 nu) i t0 + ((2 nu - 1) - zeta) t2
  v = caxpy_i(cscale(t2, (T)2 * nu - (T)1 - zeta), zeta - (T)2 * nu, t0);
  e[2] = caxpy(e[2], c2, v);
  // p3: -t1 / (2 mu) ; qp: i t1 / (2 mu)
  e[3] = caxpy(e[3], -c2, t1);
  e[5] = caxpy_i(e[5], c2, t1);
  // q3: (-t0 + zeta (t0 + i t2)) / (2 mu) = (zeta - 1) t0 + zeta i t2
  v = caxpy_i(cscale(t0, zeta - (T)1), zeta, t2);
  e[4] = caxpy(e[4], c2, v);
}

// rotate a symmetric tensor (11,22,33,23,13,12) into the (q, p, 3) frame and back
template <typename T, typename V>
__device__ __forceinline__ void rotate_in(V* x, T c, T s) {
  const V X11 = x[0], X22 = x[1], X23 = x[3], X13 = x[4], X12 = x[5];
  const T cc = c * c, ss = s * s, cs = c * s;
  x[0] = caxpy(caxpy(cscale(X11, cc), ss, X22), (T)2 * cs, X12);
  x[1] = caxpy(caxpy(cscale(X11, ss), cc, X22), (T)-2 * cs, X12);
  x[3] = caxpy(cscale(X13, -s), c, X23);
  x[4] = caxpy(cscale(X13, c), s, X23);
  x[5] = caxpy(caxpy(cscale(X11, -cs), cs, X22), cc - ss, X12);
}
template <typename T, typename V>
__device__ __forceinline__ void rotate_out(V* y, T c, T s) {
  const V qq = y[0], pp = y[1], p3 = y[3], q3 = y[4], qp = y[5];
  const T cc = c * c, ss = s * s, cs = c * s;
  y[0] = caxpy(caxpy(cscale(qq, cc), ss, pp), (T)-2 * cs, qp);
  y[1] = caxpy(caxpy(cscale(qq, ss), cc, pp), (T)2 * cs, qp);
  y[3] = caxpy(cscale(q3, s), c, p3);
  y[4] = caxpy(cscale(q3, c), -s, p3);
  y[5] = caxpy(caxpy(cscale(qq, cs), -cs, pp), cc - ss, qp);
}

template <typename T> struct ModeGeom {
  T q, c, s;
  bool zero, nyq;
};

// wavevector of the mode (k1, k2) in the arithmetic of the path: w1 = 2 pi / L1, w2 = 2 pi / L2.
// k2 is signed (k2 - N2 above N2/2); modes outside Z^2_N (k1 = N1/2 or k2 = N2/2 on even
// sides) and the padding columns k1 >= hs carry no operator term (flag nyq).
template <typename T>
__device__ __forceinline__ ModeGeom<T> mode_geom(int k1, int k2, int n1, int n2, int hs, T w1, T w2) {
  ModeGeom<T> g;
  const int k2s = 2 * k2 < n2 ? k2 : k2 - n2;
  g.nyq = (2 * k2 == n2) || (2 * k1 == n1) || k1 >= hs;
  g.zero = (k1 == 0 && k2 == 0);
  const T q1 = w1 * (T)k1;
  const T q2 = w2 * (T)k2s;
  const T q = sqrt(q1 * q1 + q2 * q2);
  const T iq = q > (T)0 ? (T)1 / q : (T)0;
  g.q = q;
  g.c = q > (T)0 ? q1 * iq : (T)1;
  g.s = q2 * iq;
  return g;
}

// ----------------------------------------------------------------------------------
// Mindlin depth kernel
// grid: (h1 / KT, n2); block: KT * nch threads, thread = (chunk, k1 column)
// smem: W[nz][6][KT] (rotated in place) + Pst[max(nz, 2 nch + 1)][6][KT]
// ----------------------------------------------------------------------------------
template <typename T, int KT, bool EIN>
__global__ void __launch_bounds__(256) k_mindlin_depth(typename Cx<T>::t* __restrict__ spec, typename Cx<T>::t* __restrict__ surf,
                                const T* __restrict__ zn, int nz, int n1, int n2, int hs, int h1, int C, int nch, int prow, T w1,
                                T w2, T lam, T mu, T nu, int out_kind, int want_u3, int uniform, T hz,
                                const int* __restrict__ zr) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(128) unsigned char smraw[];  // one alignment for every kernel of this file
  V* W = reinterpret_cast<V*>(smraw);                 // [nz][6][KT]
  V* Pst = W + (size_t)nz * 6 * KT;                   // [max(nz, 2 nch + 1)][6][KT]
  T* zs = reinterpret_cast<T*>(Pst + (size_t)prow * KT * 6);  // [nz] depth nodes
  const int kt = threadIdx.x & (KT - 1);
  const int ch = threadIdx.x / KT;
  const int k1 = blockIdx.x * KT + kt;
  const int k2 = blockIdx.y;
  const size_t plane = (size_t)n2 * h1;
  const size_t colofs = (size_t)k2 * h1 + blockIdx.x * KT;

  // 1. load the tile (coalesced KT-wide rows, every copy in flight before one wait) and
  //    the depth nodes
  // (layers outside zr hold no input: their spectrum was not computed and reads as zero)
  if (!zr) {
    for (int idx = threadIdx.x; idx < nz * 6 * KT; idx += blockDim.x) {
      const int zc = idx / KT, j = idx & (KT - 1);
      cp_async_cx(W + idx, spec + (size_t)zc * plane + colofs + j);
    }
  } else {
    const int zlo = zr[0], zhi = zr[1];
    for (int idx = threadIdx.x; idx < nz * 6 * KT; idx += blockDim.x) {
      const int zc = idx / KT, j = idx & (KT - 1);
      const int zl = zc / 6;
      if (zl >= zlo && zl < zhi) cp_async_cx(W + idx, spec + (size_t)zc * plane + colofs + j);
      else W[idx] = mk<V>(0, 0);
    }
  }
  for (int i = threadIdx.x; i < nz; i += blockDim.x) zs[i] = zn[i];
  cp_async_wait_all();
  __syncthreads();

  const ModeGeom<T> g = mode_geom<T>(k1, k2, n1, n2, hs, w1, w2);
  const bool special = g.zero || g.nyq;
  const int n0 = ch * C;
  const int nend = min(n0 + C, nz);
  const int e1 = min(n0 + C, nz - 1);  // elements [n0, e1)
  const bool active = n0 < nz;

  // 2. (eps_p input: w = C:eps_p per mode) rotate own nodes into the (q, p, 3) frame
  if (active && (EIN || !special)) {
    for (int i = n0; i < nend; ++i) {
      V x[6];
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) x[cc] = W[(i * 6 + cc) * KT + kt];
      if (EIN) {
        const V tr = cadd(cadd(x[0], x[1]), x[2]);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) x[cc] = cscale(x[cc], (T)2 * mu);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) x[cc] = caxpy(x[cc], lam, tr);
      }
      if (!special) rotate_in(x, g.c, g.s);
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) W[(i * 6 + cc) * KT + kt] = x[cc];
    }
  }
  __syncthreads();

  Elem<T> ec;
  if (uniform) ec = elem_coef<T>(g.q, hz);

  // 3. local summaries of both recursions over the chunk's elements, from zero
  Mom<V>* SP = reinterpret_cast<Mom<V>*>(Pst);          // [nch][KT]
  Mom<V>* SA = SP + (size_t)nch * KT;                   // [nch][KT]
  if (active && !special) {
    Mom<V> A, P;
    mom_zero(A);
    mom_zero(P);
    for (int e = n0; e < e1; ++e) {
      if (!uniform) ec = elem_coef<T>(g.q, zs[e + 1] - zs[e]);
      V wi[6], wj[6];
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        wi[cc] = W[(e * 6 + cc) * KT + kt];
        wj[cc] = W[((e + 1) * 6 + cc) * KT + kt];
      }
      stepA(A, ec, wi, wj);
    }
    for (int e = e1 - 1; e >= n0; --e) {
      if (!uniform) ec = elem_coef<T>(g.q, zs[e + 1] - zs[e]);
      V wi[6], wj[6];
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        wi[cc] = W[(e * 6 + cc) * KT + kt];
        wj[cc] = W[((e + 1) * 6 + cc) * KT + kt];
      }
      stepP(P, ec, wi, wj);
    }
    SA[ch * KT + kt] = A;
    SP[ch * KT + kt] = P;
  }
  __syncthreads();

  // 4. carries: A at node n0 from all chunks above, P at node e1 from all chunks below,
  //    and the complete + branch at x3 = 0 for the image term.  One exclusive scan per
  //    branch and mode (thread ch 0: downwards, thread ch 1: upwards), in place over the
  //    chunk summaries: slot j ends up holding the carry into chunk j.
  Mom<V>* P0s = SA + (size_t)nch * KT;  // [KT]
  if (active && !special) {
    const int pch = nch > 1 ? 1 : 0;
    if (ch == 0) {
      Mom<V> run;
      mom_zero(run);
      for (int j = 0; j < nch; ++j) {
        const int a0 = j * C, a1 = min(j * C + C, nz - 1);
        const Mom<V> sj = SA[j * KT + kt];
        SA[j * KT + kt] = run;
        propA(run, g.q * (zs[a1] - zs[a0]));
        mom_add(run, sj);
      }
    }
    if (ch == pch) {
      Mom<V> run;
      mom_zero(run);
      for (int j = nch - 1; j >= 0; --j) {
        const int a0 = j * C, a1 = min(j * C + C, nz - 1);
        const Mom<V> sj = SP[j * KT + kt];
        SP[j * KT + kt] = run;
        propP(run, g.q * (zs[a1] - zs[a0]));
        mom_add(run, sj);
      }
      P0s[kt] = run;
    }
  }
  __syncthreads();
  Mom<V> Ain, Pin, P0;
  if (active && !special) {
    Ain = SA[ch * KT + kt];
    Pin = SP[ch * KT + kt];
    P0 = P0s[kt];
  } else {
    mom_zero(Ain);
    mom_zero(Pin);
    mom_zero(P0);
  }
  // surface traction of the full-space field (A = 0 at x3 = 0), cancelled by the image
  V tr[3];
  if (active && !special) {
    V w0[6];
#pragma unroll
    for (int cc = 0; cc < 6; ++cc) w0[cc] = W[cc * KT + kt];
    Mom<V> Z;
    mom_zero(Z);
    V e0[6];
    kelvin_strain<T, V>(Z, P0, w0, g.q, nu, mu, e0);
    const V trc = cadd(e0[0], e0[2]);
    tr[0] = csub(cscale(e0[4], (T)2 * mu), w0[4]);
    tr[1] = csub(cscale(e0[3], (T)2 * mu), w0[3]);
    tr[2] = csub(caxpy(cscale(trc, lam), (T)2 * mu, e0[2]), w0[2]);
    if (want_u3 && ch == 0) {
      // u3(0) = N_inf[w].e3 + B^T(q, 0) t . e3 (rotated frame)
      const T K = (T)1 / ((T)8 * mu * (nu - (T)1));
      V u = caxpy(cmuli(P0.m[3]), (T)1, P0.m[1]);        // P_33 + i P_q3
      u = cadd(cscale(u, (T)2 - (T)4 * nu), P0.n);
      u = cscale(u, K);
      V ub = cscale(cmuli(tr[0]), (T)0.5 * ((T)2 * nu - (T)1));
      ub = caxpy(ub, -(nu - (T)1), tr[2]);
      u = caxpy(u, (T)1 / (g.q * mu), ub);
      surf[(size_t)k2 * h1 + k1] = u;
    }
  }
  if (want_u3 && ch == 0 && special) surf[(size_t)k2 * h1 + k1] = mk<V>(0, 0);
  __syncthreads();  // summaries are dead from here on; Pst is reused for P(i)

  if (!active) return;
  if (special) {
    for (int i = n0; i < nend; ++i) {
      V w[6], o[6];
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) w[cc] = W[(i * 6 + cc) * KT + kt];
      if (g.nyq) {
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) o[cc] = out_kind == FVIM_STRAIN ? mk<V>(0, 0) : cscale(w[cc], (T)-1);
      } else {
        // laminate: eps_33 = w_33/(lam+2mu), eps_a3 = w_a3/(2mu), eps_ab = 0
        V e[6];
        e[0] = e[1] = e[5] = mk<V>(0, 0);
        e[2] = cscale(w[2], (T)1 / (lam + (T)2 * mu));
        e[3] = cscale(w[3], (T)1 / ((T)2 * mu));
        e[4] = cscale(w[4], (T)1 / ((T)2 * mu));
        if (out_kind == FVIM_STRAIN) {
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) o[cc] = e[cc];
        } else {
          const V trc = e[2];
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) o[cc] = csub(cscale(e[cc], (T)2 * mu), w[cc]);
          o[0] = caxpy(o[0], lam, trc);
          o[1] = caxpy(o[1], lam, trc);
          o[2] = caxpy(o[2], lam, trc);
        }
      }
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) spec[(size_t)(i * 6 + cc) * plane + (size_t)k2 * h1 + k1] = o[cc];
    }
    return;
  }

  // 5. exact + branch at the chunk nodes (backward from the carry), kept in Pst
  Mom<V>* Pn = reinterpret_cast<Mom<V>*>(Pst);  // [node][KT]
  {
    Mom<V> P = Pin;
    if (e1 < nend) Pn[e1 * KT + kt] = P;   // last chunk: node nz-1 has no element below
    for (int e = e1 - 1; e >= n0; --e) {
      if (!uniform) ec = elem_coef<T>(g.q, zs[e + 1] - zs[e]);
      V wi[6], wj[6];
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) {
        wi[cc] = W[(e * 6 + cc) * KT + kt];
        wj[cc] = W[((e + 1) * 6 + cc) * KT + kt];
      }
      stepP(P, ec, wi, wj);
      Pn[e * KT + kt] = P;
    }
  }
  // 6. forward: - branch, combine, image, epilogue, rotate back, store
  {
    Mom<V> A = Ain;
    const T imu = (T)1 / mu;
    // exp(-q z_i): one exponential per chunk, then the element factor e^{-qh} per node
    // on uniform grids
    T ex = dexp<T>(-g.q * zs[n0]);
    for (int i = n0; i < nend; ++i) {
      V w[6];
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) w[cc] = W[(i * 6 + cc) * KT + kt];
      const Mom<V> P = Pn[i * KT + kt];
      V e[6];
      kelvin_strain<T, V>(A, P, w, g.q, nu, mu, e);
      if (!uniform && i > n0) ex = dexp<T>(-g.q * zs[i]);
      bous_strain_add<T, V>(tr, g.q * zs[i], ex, nu, imu, e);
      if (uniform) ex *= ec.E;
      V o[6];
      if (out_kind == FVIM_STRAIN) {
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) o[cc] = e[cc];
      } else {
        const V trc = cadd(e[0], e[2]);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) o[cc] = csub(cscale(e[cc], (T)2 * mu), w[cc]);
        o[0] = caxpy(o[0], lam, trc);
        o[1] = caxpy(o[1], lam, trc);
        o[2] = caxpy(o[2], lam, trc);
      }
      rotate_out(o, g.c, g.s);
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) spec[(size_t)(i * 6 + cc) * plane + (size_t)k2 * h1 + k1] = o[cc];
      if (i < e1) {
        if (!uniform) ec = elem_coef<T>(g.q, zs[i + 1] - zs[i]);
        V wj[6];
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) wj[cc] = W[((i + 1) * 6 + cc) * KT + kt];
        stepA(A, ec, w, wj);
      }
    }
  }
}

// ----------------------------------------------------------------------------------
// Mindlin depth kernel, register variant (C <= 8 nodes per chunk, compile time).  The
// summary pass keeps the + branch of the chunk's own elements per node in registers, so
// the final pass adds the propagated carry (one propagation per node) instead of running
// the + recursion again, and every pass reads each node of the tile once (the other node
// of an element is carried in registers).
// smem: W[nz][6][KT] + SA[nch][KT] + SP[nch][KT] (moments) + TR[KT][3] + zs[nz]
// ----------------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ void ld6(V (&w)[6], const V* W, int node, int KT, int kt) {
#pragma unroll
  for (int cc = 0; cc < 6; ++cc) w[cc] = W[(node * 6 + cc) * KT + kt];
}

// Per-column quantities that do not depend on the tile, computed while its copy is in flight:
// the mode geometry (every thread) and, on a uniform grid, the element integrals (one thread
// per column, written to the traction area TR as [6][KT] values of T for the body to read
// after its first barrier).
template <typename T, int KT>
__device__ __forceinline__ ModeGeom<T> depth_prep(typename Cx<T>::t* TR, int tid, int kblk, int k2, bool ghost,
                                                  int n1, int n2, int hs, T w1, T w2, int uniform, T hz) {
  const int kt = tid & (KT - 1);
  const ModeGeom<T> g = mode_geom<T>(kblk * KT + kt, k2, n1, n2, hs, w1, w2);
  if (uniform && tid < KT && !ghost) {
    T* ecs = reinterpret_cast<T*>(TR);
    const Elem<T> e = elem_coef<T>(g.q, hz);
    ecs[0 * KT + kt] = e.E;
    ecs[1 * KT + kt] = e.a;
    ecs[2 * KT + kt] = e.hI0mI1;
    ecs[3 * KT + kt] = e.hI1;
    ecs[4 * KT + kt] = e.ahI1mI2;
    ecs[5 * KT + kt] = e.ahI2;
  }
  return g;
}

// Steps 2-5 of the register depth kernel on a tile already in shared memory: W[nz][6][KT]
// (the tile), SA / SP [>= nch][KT] (chunk moments), TR[KT][3], zs[nz].  tid = ch * KT + kt is
// the thread's place in the tile, kblk the tile's block of KT k1 columns.  A ghost tile (a
// CTA slot without a tile) takes part in the barriers only.
template <typename T, int KT, int C, bool EIN>
__device__ __forceinline__ void depth_r_body(typename Cx<T>::t* W, Mom<typename Cx<T>::t>* SA,
                                             Mom<typename Cx<T>::t>* SP, typename Cx<T>::t* TR, const T* zs, int tid,
                                             int kblk, int k2, bool ghost, typename Cx<T>::t* __restrict__ spec,
                                             typename Cx<T>::t* __restrict__ surf, int nz, int n1, int n2, int hs,
                                             int h1, int nch, T w1, T w2, T lam, T mu, T nu, int out_kind,
                                             int want_u3, int uniform, T hz, T cut, const ModeGeom<T> g) {
  typedef typename Cx<T>::t V;
  const int kt = tid & (KT - 1);
  const int ch = tid / KT;
  const int k1 = kblk * KT + kt;
  const size_t plane = (size_t)n2 * h1;
  const bool special = g.zero || g.nyq;
  const int n0 = ch * C;
  const int nend = min(n0 + C, nz);
  const int e1 = min(n0 + C, nz - 1);  // elements [n0, e1)
  const bool active = !ghost && n0 < nz;
  const bool work = active && !special;

  // 2. (eps_p input: w = C:eps_p per mode) rotate own nodes into the (q, p, 3) frame
  if (active) {
#pragma unroll
    for (int l = 0; l < C; ++l) {
      const int i = n0 + l;
      if (i >= nend) break;
      V x[6];
      ld6(x, W, i, KT, kt);
      if (EIN) {
        const V tr = cadd(cadd(x[0], x[1]), x[2]);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) x[cc] = cscale(x[cc], (T)2 * mu);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) x[cc] = caxpy(x[cc], lam, tr);
      }
      if (!special) rotate_in(x, g.c, g.s);
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) W[(i * 6 + cc) * KT + kt] = x[cc];
    }
  }
  // element coefficients of a uniform grid: the chunk threads of a column share q and h, so
  // one thread per column evaluated them (depth_prep, before this barrier) and the others read
  // them here.  They pass through the traction area TR ([6][KT] values of T), which is written
  // again only after later barriers, when every thread holds them in registers.
  const T* ecs = reinterpret_cast<const T*>(TR);
  __syncthreads();

  Elem<T> ec;
  if (uniform) {
    ec.E = ecs[0 * KT + kt];
    ec.a = ecs[1 * KT + kt];
    ec.h = hz;
    ec.hI0mI1 = ecs[2 * KT + kt];
    ec.hI1 = ecs[3 * KT + kt];
    ec.ahI1mI2 = ecs[4 * KT + kt];
    ec.ahI2 = ecs[5 * KT + kt];
  }

  // 3. chunk summaries from zero (- branch at the chunk's last node e1, + branch at its
  //    first node n0); the + branch of every own node stays in registers
  Mom<V> Ploc[C];
  Mom<V> Ta, Up;
  mom_zero(Ta);
  mom_zero(Up);
  if (work && uniform) {
    // the two recursions are independent chains: advance them together (same steps in the
    // same order per chain as below, so the same values)
    V wa[6], wb[6];
    ld6(wa, W, n0, KT, kt);
    ld6(wb, W, e1, KT, kt);
#pragma unroll
    for (int st = 0; st < C; ++st) {
      const int la = st, lp = C - 1 - st;
      if (n0 + la < e1) {
        V wn[6];
        ld6(wn, W, n0 + la + 1, KT, kt);
        stepA(Ta, ec, wa, wn);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) wa[cc] = wn[cc];
      }
      if (n0 + lp < e1) {
        V wc[6];
        ld6(wc, W, n0 + lp, KT, kt);
        stepP(Up, ec, wc, wb);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) wb[cc] = wc[cc];
        Ploc[lp] = Up;
      } else {
        mom_zero(Ploc[lp]);
      }
    }
  } else if (work) {
    V wa[6];
    ld6(wa, W, n0, KT, kt);
#pragma unroll
    for (int l = 0; l < C; ++l) {
      const int e = n0 + l;
      if (e < e1) {
        if (!uniform) ec = elem_coef<T>(g.q, zs[e + 1] - zs[e]);
        V wb[6];
        ld6(wb, W, e + 1, KT, kt);
        stepA(Ta, ec, wa, wb);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) wa[cc] = wb[cc];
      }
    }
    V wb[6];
    ld6(wb, W, e1, KT, kt);
#pragma unroll
    for (int l = C - 1; l >= 0; --l) {
      const int e = n0 + l;
      if (e < e1) {
        if (!uniform) ec = elem_coef<T>(g.q, zs[e + 1] - zs[e]);
        V wc[6];
        ld6(wc, W, e, KT, kt);
        stepP(Up, ec, wc, wb);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) wb[cc] = wc[cc];
        Ploc[l] = Up;
      } else {
        mom_zero(Ploc[l]);
      }
    }
  }

  // 4. inclusive scans over the chunks, log2(nch) rounds with every chunk thread working:
  //    - branch downwards, Ta_j = sum_{i<=j} propA(S_i, q (z[e1_j] - z[e1_i]));
  //    + branch upwards,  Up_j = sum_{i>=j} propP(S_i, q (z[n0_i] - z[n0_j])).
  //    Propagations compose (prop(prop(M, a), b) = prop(M, a + b)), so the rounds are exact.
  // Cutoff (Sec. 3.2, eps_co, restated for the recursion): when every chunk span of the tile
  // damps by e^{-q span} < e^{-cut}, a chunk's carry is its neighbour's own summary to the
  // rounding of the path (e^{-18} < 2^-24 in FP32): the chunks beyond the neighbour contribute
  // below it, so the scan rounds are skipped (one block-wide vote keeps the branch uniform)
  const T span = (work && ch + 1 < nch) ? zs[e1] - zs[n0] : (T)0;
  const bool far = !work || ch + 1 >= nch || g.q * span > cut;
  const bool local = __syncthreads_and(cut > (T)0 && far) != 0;
  const int e1c = e1;
  for (int d = 1; d < nch && !local; d <<= 1) {
    SA[ch * KT + kt] = Ta;
    SP[ch * KT + kt] = Up;
    __syncthreads();
    if (work && ch >= d) {
      Mom<V> o = SA[(ch - d) * KT + kt];
      const int e1o = min((ch - d) * C + C, nz - 1);
      propA(o, g.q * (zs[e1c] - zs[e1o]));
      mom_add(Ta, o);
    }
    if (work && ch + d < nch) {
      Mom<V> o = SP[(ch + d) * KT + kt];
      propP(o, g.q * (zs[(ch + d) * C] - zs[n0]));
      mom_add(Up, o);
    }
    __syncthreads();
  }
  SA[ch * KT + kt] = Ta;
  SP[ch * KT + kt] = Up;
  __syncthreads();

  // surface traction of the full-space field (A = 0 at x3 = 0, + branch complete: the
  // scan value of chunk 0), cancelled by the image; one thread per column, the last chunk's
  // (it has no carry from below to fold, so it works while the other chunks fold theirs)
  const int tch = nch - 1;
  if (ch == tch && work) {
    V w0[6];
    ld6(w0, W, 0, KT, kt);
    const Mom<V> U0 = SP[kt];
    Mom<V> Z;
    mom_zero(Z);
    V e0[6];
    kelvin_strain<T, V>(Z, U0, w0, g.q, nu, mu, e0);
    const V trc = cadd(e0[0], e0[2]);
    const V t0 = csub(cscale(e0[4], (T)2 * mu), w0[4]);
    const V t1 = csub(cscale(e0[3], (T)2 * mu), w0[3]);
    const V t2 = csub(caxpy(cscale(trc, lam), (T)2 * mu, e0[2]), w0[2]);
    TR[3 * kt] = t0;
    TR[3 * kt + 1] = t1;
    TR[3 * kt + 2] = t2;
    if (want_u3) {
      // u3(0) = N_inf[w].e3 + B^T(q, 0) t . e3 (rotated frame)
      const T K = (T)1 / ((T)8 * mu * (nu - (T)1));
      V u = caxpy(cmuli(U0.m[3]), (T)1, U0.m[1]);  // P_33 + i P_q3
      u = cadd(cscale(u, (T)2 - (T)4 * nu), U0.n);
      u = cscale(u, K);
      V ub = cscale(cmuli(t0), (T)0.5 * ((T)2 * nu - (T)1));
      ub = caxpy(ub, -(nu - (T)1), t2);
      u = caxpy(u, (T)1 / (g.q * mu), ub);
      surf[(size_t)k2 * h1 + k1] = u;
    }
  }
  if (want_u3 && ch == tch && special) surf[(size_t)k2 * h1 + k1] = mk<V>(0, 0);
  // the carry from below folded into the per-node + branch (so that it is not live during
  // the output loop)
  if (work && ch + 1 < nch) {
    const Mom<V> Pin = SP[(ch + 1) * KT + kt];
    if (uniform) {
      // a chunk above the last one is whole (e1 = n0 + C): node n0 + l lies C - l elements
      // above e1, so its propagator is E^(C - l), built by products
      T Ek = ec.E;
#pragma unroll
      for (int l = C - 1; l >= 0; --l) {
        Mom<V> P = Pin;
        propP_E(P, g.q * hz * (T)(C - l), Ek);
        mom_add(Ploc[l], P);
        Ek *= ec.E;
      }
    } else {
#pragma unroll
      for (int l = 0; l < C; ++l) {
        if (n0 + l < nend) {
          Mom<V> P = Pin;
          propP(P, g.q * (zs[e1] - zs[n0 + l]));
          mom_add(Ploc[l], P);
        }
      }
    }
  }
  __syncthreads();

  if (!active) return;
  if (special) {
    for (int i = n0; i < nend; ++i) {
      V w[6], o[6];
      ld6(w, W, i, KT, kt);
      if (g.nyq) {
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) o[cc] = out_kind == FVIM_STRAIN ? mk<V>(0, 0) : cscale(w[cc], (T)-1);
      } else {
        // laminate: eps_33 = w_33/(lam+2mu), eps_a3 = w_a3/(2mu), eps_ab = 0
        V e[6];
        e[0] = e[1] = e[5] = mk<V>(0, 0);
        e[2] = cscale(w[2], (T)1 / (lam + (T)2 * mu));
        e[3] = cscale(w[3], (T)1 / ((T)2 * mu));
        e[4] = cscale(w[4], (T)1 / ((T)2 * mu));
        if (out_kind == FVIM_STRAIN) {
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) o[cc] = e[cc];
        } else {
          const V trc = e[2];
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) o[cc] = csub(cscale(e[cc], (T)2 * mu), w[cc]);
          o[0] = caxpy(o[0], lam, trc);
          o[1] = caxpy(o[1], lam, trc);
          o[2] = caxpy(o[2], lam, trc);
        }
      }
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) spec[(size_t)(i * 6 + cc) * plane + (size_t)k2 * h1 + k1] = o[cc];
    }
    return;
  }

  // 5. forward over the chunk: - branch from its carry (scan value of the chunk above),
  //    + branch = own part + carry from below (folded above), image term, epilogue, rotate
  //    back, store
  Mom<V> A;
  if (ch > 0) A = SA[(ch - 1) * KT + kt];
  else mom_zero(A);
  V tr[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) tr[j] = TR[3 * kt + j];
  const T imu = (T)1 / mu;
  T ex = dexp<T>(-g.q * zs[n0]);
  V w[6];
  ld6(w, W, n0, KT, kt);
#pragma unroll
  for (int l = 0; l < C; ++l) {
    const int i = n0 + l;
    if (i < nend) {
      const Mom<V>& P = Ploc[l];
      V e[6];
      kelvin_strain<T, V>(A, P, w, g.q, nu, mu, e);
      if (!uniform && l > 0) ex = dexp<T>(-g.q * zs[i]);
      bous_strain_add<T, V>(tr, g.q * zs[i], ex, nu, imu, e);
      if (uniform) ex *= ec.E;
      V o[6];
      if (out_kind == FVIM_STRAIN) {
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) o[cc] = e[cc];
      } else {
        const V trc = cadd(e[0], e[2]);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) o[cc] = csub(cscale(e[cc], (T)2 * mu), w[cc]);
        o[0] = caxpy(o[0], lam, trc);
        o[1] = caxpy(o[1], lam, trc);
        o[2] = caxpy(o[2], lam, trc);
      }
      rotate_out(o, g.c, g.s);
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) spec[(size_t)(i * 6 + cc) * plane + (size_t)k2 * h1 + k1] = o[cc];
      if (i < e1) {
        if (!uniform) ec = elem_coef<T>(g.q, zs[i + 1] - zs[i]);
        V wj[6];
        ld6(wj, W, i + 1, KT, kt);
        stepA(A, ec, w, wj);
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) w[cc] = wj[cc];
      }
    }
  }
}

template <typename T, int KT, int C, bool EIN, int MB>
__global__ void __launch_bounds__(256, MB) k_mindlin_depth_r(typename Cx<T>::t* __restrict__ spec,
                                                            typename Cx<T>::t* __restrict__ surf,
                                                            const T* __restrict__ zn, int nz, int n1, int n2, int hs, int h1, int nch,
                                                            T w1, T w2, T lam, T mu, T nu, int out_kind, int want_u3,
                                                            int uniform, T hz, const int* __restrict__ zr, T cut,
                                                            const __grid_constant__ CUtensorMap tmap, int tma_rows,
                                                            int tx_extra, int* __restrict__ status) {
  typedef typename Cx<T>::t V;
  static_assert(sizeof(V) == 8 && KT % 2 == 0, "FP32 tiles of an even width");
  extern __shared__ __align__(128) unsigned char smraw[];  // tensor-copy boxes land at 128-byte offsets
  V* W = reinterpret_cast<V*>(smraw);                               // [nz][6][KT]
  Mom<V>* SA = reinterpret_cast<Mom<V>*>(W + (size_t)nz * 6 * KT);  // [nch][KT]
  Mom<V>* SP = SA + (size_t)nch * KT;                               // [nch][KT]
  V* TR = reinterpret_cast<V*>(SP + (size_t)nch * KT);              // [KT][3] image traction
  T* zs = reinterpret_cast<T*>(TR + 3 * KT);                        // [nz]
  // mbarrier of the tensor copies, 8-byte aligned after the depth nodes
  unsigned long long* tbar = reinterpret_cast<unsigned long long*>(
      reinterpret_cast<unsigned char*>(zs) + (((size_t)nz * sizeof(T) + 7) & ~(size_t)7));
  const int k2 = blockIdx.y;
  const size_t plane = (size_t)n2 * h1;
  const size_t colofs = (size_t)k2 * h1 + blockIdx.x * KT;
  ModeGeom<T> g;

  // 1. load the tile and the depth nodes (layers outside zr hold no input: their spectrum was
  //    not computed and reads as zero).  With a tensor map (tma_rows > 0): one thread issues
  //    tensor copies of tma_rows x KT complex boxes (rows z c, one k2, KT columns) that complete
  //    on an mbarrier; the wait is bounded, and a copy that never completes sets the status word
  //    and every thread of the CTA returns after a second bounded wait.  Otherwise 16-byte
  //    cp.async copies by all threads.
  if (tma_rows > 0) {
    const unsigned bar = (unsigned)__cvta_generic_to_shared(tbar);
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned bytes = (unsigned)(nz * 6 * KT * sizeof(V) + tx_extra);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
      const int x = (int)(blockIdx.x * KT * 2);  // first k1 column, in floats (16-byte multiple)
      for (int r0 = 0; r0 < nz * 6; r0 += tma_rows) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(W + (size_t)r0 * KT);
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(dst),
            "l"(reinterpret_cast<unsigned long long>(&tmap)), "r"(x), "r"(k2), "r"(r0), "r"(bar)
            : "memory");
      }
    }
    for (int i = threadIdx.x; i < nz; i += blockDim.x) zs[i] = zn[i];
    g = depth_prep<T, KT>(TR, threadIdx.x, blockIdx.x, k2, false, n1, n2, hs, w1, w2, uniform, hz);
    bool done = mbar_wait_bounded(bar, 1000000000ull);   // 1 s
    if (__syncthreads_or(!done)) {
      if (threadIdx.x == 0 && status) atomicOr(status, 1);
      if (!done) mbar_wait_bounded(bar, 1000000000ull);  // the copies of this CTA, once more
      return;
    }
    if (zr) {
      const int zlo = zr[0], zhi = zr[1];
      for (int idx = threadIdx.x; idx < nz * 6 * KT; idx += blockDim.x) {
        const int zl = idx / (6 * KT);
        if (zl < zlo || zl >= zhi) W[idx] = mk<V>(0, 0);
      }
    }
    __syncthreads();
  } else if (!zr) {
    for (int idx = threadIdx.x; idx < nz * 6 * (KT / 2); idx += blockDim.x) {
      const int zc = idx / (KT / 2), j = 2 * (idx % (KT / 2));
      cp_async_16(W + zc * KT + j, spec + (size_t)zc * plane + colofs + j);
    }
  } else {
    const int zlo = zr[0], zhi = zr[1];
    for (int idx = threadIdx.x; idx < nz * 6 * (KT / 2); idx += blockDim.x) {
      const int zc = idx / (KT / 2), j = 2 * (idx % (KT / 2));
      const int zl = zc / 6;
      if (zl >= zlo && zl < zhi) {
        cp_async_16(W + zc * KT + j, spec + (size_t)zc * plane + colofs + j);
      } else {
        W[zc * KT + j] = mk<V>(0, 0);
        W[zc * KT + j + 1] = mk<V>(0, 0);
      }
    }
  }
  if (tma_rows <= 0) {
    for (int i = threadIdx.x; i < nz; i += blockDim.x) zs[i] = zn[i];
    g = depth_prep<T, KT>(TR, threadIdx.x, blockIdx.x, k2, false, n1, n2, hs, w1, w2, uniform, hz);
    cp_async_wait_all();
    __syncthreads();
  }

  depth_r_body<T, KT, C, EIN>(W, SA, SP, TR, zs, threadIdx.x, blockIdx.x, k2, false, spec, surf, nz, n1, n2, hs, h1,
                              nch, w1, w2, lam, mu, nu, out_kind, want_u3, uniform, hz, cut, g);
}

// ----------------------------------------------------------------------------------
// Grouped depth kernel: the tiles of every problem of a GrpTable in one launch.  Chunks of 4
// nodes, 16-column tiles; a CTA of 256 threads holds 16 / nchp tiles of one problem (nchp:
// the chunk count rounded up to a power of two; the chunks beyond nch have no nodes), each
// with its own shared-memory slot, loaded with 16-byte cp.async copies.  The cutoff vote is
// taken over the CTA's tiles together.
// ----------------------------------------------------------------------------------
__host__ __device__ constexpr size_t grp_depth_slot(int nz, int nchp) {
  return (size_t)nz * 6 * 16 * sizeof(float2) + (size_t)2 * nchp * 16 * sizeof(Mom<float2>) +
         (size_t)3 * 16 * sizeof(float2) + (((size_t)nz * sizeof(float) + 15) & ~(size_t)15);
}

__global__ void __launch_bounds__(256, 2) k_grp_depth(const __grid_constant__ GrpTable tab) {
  typedef float2 V;
  constexpr int KT = 16, C = 4;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int pi = grp_find(tab, blockIdx.x);
  const GrpProb& P = tab.p[pi];
  const int nz = P.nz, nchp = P.nchp, tt = KT * nchp, tpc = 256 / tt;
  const int j = threadIdx.x / tt, tid = threadIdx.x - j * tt;
  const int ncb = P.h1 / KT, tiles = ncb * P.n2;
  const int tile = ((int)blockIdx.x - tab.start[pi]) * tpc + j;
  const bool ghost = tile >= tiles;
  const int kblk = ghost ? 0 : tile % ncb, k2 = ghost ? 0 : tile / ncb;
  unsigned char* base = smraw + (size_t)j * grp_depth_slot(nz, nchp);
  V* W = reinterpret_cast<V*>(base);                                // [nz][6][KT]
  Mom<V>* SA = reinterpret_cast<Mom<V>*>(W + (size_t)nz * 6 * KT);  // [nchp][KT]
  Mom<V>* SP = SA + (size_t)nchp * KT;                              // [nchp][KT]
  V* TR = reinterpret_cast<V*>(SP + (size_t)nchp * KT);             // [KT][3]
  float* zs = reinterpret_cast<float*>(TR + 3 * KT);                // [nz]
  if (!ghost) {
    const size_t plane = (size_t)P.n2 * P.h1;
    const size_t colofs = (size_t)k2 * P.h1 + (size_t)kblk * KT;
    for (int idx = tid; idx < nz * 6 * (KT / 2); idx += tt) {
      const int zc = idx / (KT / 2), jj = 2 * (idx % (KT / 2));
      cp_async_16(W + zc * KT + jj, P.spec + (size_t)zc * plane + colofs + jj);
    }
    for (int i = tid; i < nz; i += tt) zs[i] = P.zn[i];
  }
  const ModeGeom<float> g =
      depth_prep<float, KT>(TR, tid, kblk, k2, ghost, P.n1, P.n2, P.hs, P.w1, P.w2, P.uniform, P.hz);
  cp_async_wait_all();
  __syncthreads();
  depth_r_body<float, KT, C, false>(W, SA, SP, TR, zs, tid, kblk, k2, ghost, P.spec, nullptr, nz, P.n1, P.n2, P.hs,
                                    P.h1, P.nch, P.w1, P.w2, P.lam, P.mu, P.nu, P.out_kind, 0, P.uniform, P.hz,
                                    P.cut, g);
}

// ----------------------------------------------------------------------------------
// Boussinesq operator of a normal pressure (Eq. B:fourier): one thread per mode, loop
// over depth.  surf holds p_hat on entry and u3_hat = 2 p_hat / (E* q) on exit.
// ----------------------------------------------------------------------------------
template <typename T>
__global__ void k_boussinesq(typename Cx<T>::t* __restrict__ spec, typename Cx<T>::t* __restrict__ surf,
                             const T* __restrict__ zn, int nz, int n1, int n2, int hs, int h1, T w1, T w2, T lam,
                             T mu, T nu, int out_kind, int want_vol, int want_u3) {
  typedef typename Cx<T>::t V;
  const int k1 = blockIdx.x * blockDim.x + threadIdx.x;
  const int k2 = blockIdx.y;
  if (k1 >= h1) return;
  const ModeGeom<T> g = mode_geom<T>(k1, k2, n1, n2, hs, w1, w2);
  const size_t plane = (size_t)n2 * h1;
  const size_t at = (size_t)k2 * h1 + k1;
  const V p = surf[at];
  if (want_vol) {
    for (int i = 0; i < nz; ++i) {
      V o[6];
      if (g.nyq) {
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) o[cc] = mk<V>(0, 0);
      } else if (g.zero) {
        const V e33 = cscale(p, (T)-1 / (lam + (T)2 * mu));
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) o[cc] = mk<V>(0, 0);
        if (out_kind == FVIM_STRAIN) {
          o[2] = e33;
        } else {
          o[0] = o[1] = cscale(e33, lam);
          o[2] = cscale(p, (T)-1);
        }
      } else {
        V e[6];
#pragma unroll
        for (int cc = 0; cc < 6; ++cc) e[cc] = mk<V>(0, 0);
        V tr[3] = {mk<V>(0, 0), mk<V>(0, 0), p};
        bous_strain_add<T, V>(tr, g.q * zn[i], dexp<T>(-g.q * zn[i]), nu, (T)1 / mu, e);
        if (out_kind == FVIM_STRAIN) {
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) o[cc] = e[cc];
        } else {
          const V trc = cadd(e[0], e[2]);
#pragma unroll
          for (int cc = 0; cc < 6; ++cc) o[cc] = cscale(e[cc], (T)2 * mu);
          o[0] = caxpy(o[0], lam, trc);
          o[1] = caxpy(o[1], lam, trc);
          o[2] = caxpy(o[2], lam, trc);
        }
        rotate_out(o, g.c, g.s);
      }
#pragma unroll
      for (int cc = 0; cc < 6; ++cc) spec[(size_t)(i * 6 + cc) * plane + at] = o[cc];
    }
  }
  if (want_u3) {
    V u = mk<V>(0, 0);
    if (!g.zero && !g.nyq) u = cscale(p, ((T)1 - nu) / (mu * g.q));
    surf[at] = u;
  }
}

}  // namespace

// Launch configuration of the depth kernel for chunk length C (nodes per chunk thread).
// Every valid C gives the same operator up to the rounding order of the chunk scan.
template <typename T> struct DepthCfg {
  bool ok;        // launchable (threads, shared memory)
  bool reg;       // FP32 register variant
  int C, nch, KT, threads;
  size_t smem;
  int mb;         // register variant: CTAs per SM it is compiled for (2: 128 registers, 3: 85)
};

int depth_chunk_default(int nz) {
  const int C = (nz + 15) / 16;
  return C < 2 ? 2 : C;
}

template <typename T> DepthCfg<T> depth_cfg(const fvim_ctx* c, int C, int ctas) {
  typedef typename Cx<T>::t V;
  DepthCfg<T> d{};
  const int nz = c->nz, h1 = c->h1;
  d.ok = false;
  if (C < 2 || C > nz) return d;
  if constexpr (sizeof(T) == 4) {
    // FP32, 16-column tiles, at most 8 nodes per chunk: the register variant (C rounded up
    // to an instantiated chunk length)
    if (h1 >= KT_MAX && C <= 8) {
      const int CR = C <= 2 ? 2 : (C <= 3 ? 3 : (C <= 4 ? 4 : (C <= 6 ? 6 : 8)));
      const int nchr = (nz + CR - 1) / CR;
      const size_t smr = (size_t)nz * 6 * 16 * sizeof(V) + (size_t)(2 * nchr) * 16 * sizeof(Mom<V>) +
                         (size_t)3 * 16 * sizeof(V) + (((size_t)nz * sizeof(T) + 7) & ~(size_t)7) + 16;
      if (smr <= 227 * 1024 && 16 * nchr <= 256) {
        // three CTAs per SM (85 registers): chunk lengths 4..8 whose tile fits three times
        if (ctas == 3 && !(CR >= 4 && 3 * (smr + 1024) <= 228 * 1024)) return d;
        d = DepthCfg<T>{true, true, CR, nchr, 16, 16 * nchr, smr, ctas == 3 ? 3 : 2};
        return d;
      }
    }
  }
  if (ctas == 3) return d;  // the shared-memory variant has one launch shape per chunk length
  const int nch = (nz + C - 1) / C;
  const int prow = nz > 2 * nch + 1 ? nz : 2 * nch + 1;
  // tile width: 16 k1 columns (128-byte rows in FP32), narrower where the depth column of
  // the tile does not fit in shared memory (deep grids, FP64)
  int KT = h1 < KT_MAX ? h1 : KT_MAX;  // h1 is a power of two
  auto smem_of = [&](int kt) {
    return (size_t)nz * 6 * kt * sizeof(V) + (size_t)prow * kt * sizeof(Mom<V>) + (size_t)nz * sizeof(T);
  };
  while (KT > 2 && smem_of(KT) > 227 * 1024) KT >>= 1;
  d.C = C;
  d.nch = nch;
  d.KT = KT;
  d.threads = KT * nch;
  d.smem = smem_of(KT);
  d.reg = false;
  d.ok = d.smem <= 227 * 1024 && d.threads <= 256;
  return d;
}

int depth_launch_ctas(const fvim_ctx* c) {
  const int C = c->depth_chunk > 0 ? c->depth_chunk : depth_chunk_default(c->nz);
  if (c->prec == FVIM_FP64) return 0;
  const DepthCfg<float> d = depth_cfg<float>(c, C, c->depth_ctas);
  return d.ok && d.reg ? d.mb : 0;
}

bool depth_chunk_ok(const fvim_ctx* c, int C, int ctas) {
  return c->prec == FVIM_FP64 ? depth_cfg<double>(c, C, ctas).ok : depth_cfg<float>(c, C, ctas).ok;
}

template <typename T>
int launch_mindlin_depth(const fvim_ctx* c, int out_kind, bool want_u3, bool eps_in, const int* zr) {
  typedef typename Cx<T>::t V;
  const int nz = c->nz, h1 = c->h1, n2 = c->n2;
  const DepthCfg<T> d = depth_cfg<T>(c, c->depth_chunk > 0 ? c->depth_chunk : depth_chunk_default(nz), c->depth_ctas);
  if (!d.ok) return FVIM_ERR_UNSUPPORTED;
  const int KT = d.KT, C = d.C, nch = d.nch;
  const int prow = nz > 2 * nch + 1 ? nz : 2 * nch + 1;
  dim3 grid(h1 / KT, n2);
  const T w1 = (T)(kTwoPi / c->L1), w2 = (T)(kTwoPi / c->L2);
  if constexpr (sizeof(T) == 4) if (d.reg) {
    // tensor-map copies of the tile where the context has its map (rows per box divide 6 Nz)
    CUtensorMap tm;
    int tma_rows = 0;
    if (c->tmap && c->tma_rows > 0) {
      tm = *reinterpret_cast<const CUtensorMap*>(c->tmap);
      tma_rows = c->tma_rows;
    } else {
      memset(&tm, 0, sizeof(tm));
    }
#define DEPTHR(CV, EI, MBV)                                                                                     \
  if (C == CV && eps_in == EI && d.mb == MBV) {                                                                 \
    smem_cap(k_mindlin_depth_r<T, 16, CV, EI, MBV>);                                                            \
    k_mindlin_depth_r<T, 16, CV, EI, MBV><<<grid, d.threads, d.smem, c->stream>>>(                              \
        (V*)c->spec, (V*)c->surf, (const T*)c->z_dev, nz, c->n1, n2, c->hs, h1, nch, w1, w2, (T)c->lam, (T)c->mu, \
        (T)c->nu,                                                                                              \
        out_kind, want_u3 ? 1 : 0, c->uniform, (T)c->hz, zr, (T)c->depth_cut, tm, tma_rows, c->tma_test_extra,  \
        c->dev_status);                                                                                          \
  }
    DEPTHR(2, false, 2) DEPTHR(3, false, 2) DEPTHR(4, false, 2) DEPTHR(6, false, 2) DEPTHR(8, false, 2)
    DEPTHR(2, true, 2) DEPTHR(3, true, 2) DEPTHR(4, true, 2) DEPTHR(6, true, 2) DEPTHR(8, true, 2)
    DEPTHR(4, false, 3) DEPTHR(6, false, 3) DEPTHR(8, false, 3)
    DEPTHR(4, true, 3) DEPTHR(6, true, 3) DEPTHR(8, true, 3)
#undef DEPTHR
    FVIM_CUDA_CHECK_LAUNCH();
    return FVIM_OK;
  }
#define DEPTH(KTV, EI)                                                                                         \
  if (KT == KTV && eps_in == EI) {                                                                             \
    smem_cap(k_mindlin_depth<T, KTV, EI>);                                                                     \
    k_mindlin_depth<T, KTV, EI><<<grid, d.threads, d.smem, c->stream>>>(                                       \
        (V*)c->spec, (V*)c->surf, (const T*)c->z_dev, nz, c->n1, n2, c->hs, h1, C, nch, prow, w1, w2, (T)c->lam,  \
        (T)c->mu,                                                                                              \
        (T)c->nu, out_kind, want_u3 ? 1 : 0, c->uniform, (T)c->hz, zr);                                       \
  }
  DEPTH(16, false) DEPTH(8, false) DEPTH(4, false) DEPTH(2, false)
  DEPTH(16, true) DEPTH(8, true) DEPTH(4, true) DEPTH(2, true)
#undef DEPTH
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

template <typename T> int launch_boussinesq(const fvim_ctx* c, int out_kind, bool want_vol, bool want_u3) {
  typedef typename Cx<T>::t V;
  const int threads = 128;
  dim3 grid((c->h1 + threads - 1) / threads, c->n2);
  k_boussinesq<T><<<grid, threads, 0, c->stream>>>((V*)c->spec, (V*)c->surf, (const T*)c->z_dev, c->nz, c->n1, c->n2,
                                                   c->hs, c->h1,
                                                   (T)(kTwoPi / c->L1), (T)(kTwoPi / c->L2), (T)c->lam, (T)c->mu, (T)c->nu,
                                                   out_kind, want_vol ? 1 : 0, want_u3 ? 1 : 0);
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

template int launch_mindlin_depth<float>(const fvim_ctx*, int, bool, bool, const int*);
template int launch_mindlin_depth<double>(const fvim_ctx*, int, bool, bool, const int*);
template int launch_boussinesq<float>(const fvim_ctx*, int, bool, bool);
template int launch_boussinesq<double>(const fvim_ctx*, int, bool, bool);

int launch_grp_depth(GrpTable& t, cudaStream_t s) {
  int b = 0;
  size_t smem = 0;
  for (int i = 0; i < t.n; ++i) {
    const GrpProb& P = t.p[i];
    const int tpc = 16 / P.nchp, tiles = (P.h1 / 16) * P.n2;
    t.start[i] = b;
    b += (tiles + tpc - 1) / tpc;
    smem = std::max(smem, (size_t)tpc * grp_depth_slot(P.nz, P.nchp));
  }
  t.start[t.n] = b;
  if (b == 0) return FVIM_OK;
  smem_cap(k_grp_depth);
  k_grp_depth<<<b, 256, smem, s>>>(t);
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

// Compile-time-length variants of the register-resident in-plane FFT kernels (fft.cu has
// the runtime-length ones).  Same data layouts, same arithmetic, same results up to the
// order of operations inside the butterflies; chosen by the launchers for 16 <= N <= 1024.
#include <algorithm>

#include "fvim_internal.cuh"

namespace {

template <typename T>
__device__ __forceinline__ void hooke6_ct(const T* e, T* w, T lam, T mu) {
  const T tr = e[0] + e[1] + e[2];
  w[0] = lam * tr + 2 * mu * e[0];
  w[1] = lam * tr + 2 * mu * e[1];
  w[2] = lam * tr + 2 * mu * e[2];
  w[3] = 2 * mu * e[3];
  w[4] = 2 * mu * e[4];
  w[5] = 2 * mu * e[5];
}

// interleaved columns: entry p of column f at buf[p * KC + f]
template <typename V> struct ColSm {
  V* buf;
  int kc, f;
  __device__ __forceinline__ void put(int, int p, V x) const { buf[p * kc + f] = x; }
  __device__ __forceinline__ V get(int, int p) const { return buf[p * kc + f]; }
};
// Row exchange layout: transform g of a row at buf[g * LD + idx(p)].  8-byte entries on rows
// of 128 or more: no padding, entry p at p ^ ((p >> 3) & 15) (a permutation inside each
// aligned block of 16), so that a half-warp's accesses of the radix-8 stage writes (stride 8)
// and of the contiguous reads both fall on 16 distinct bank pairs; otherwise one pad slot
// every 8 entries (p + p / 8), which leaves the contiguous 8-byte reads two-way conflicted
// but suits 16-byte entries and rows shorter than a half-warp.
template <typename V, int N> struct RowLayout {
  static constexpr bool swz = sizeof(V) == 8 && N >= 128;
  static constexpr int LD = swz ? N : N + N / 8;
  static __device__ __forceinline__ int idx(int p) { return swz ? (p ^ ((p >> 3) & 15)) : p + (p >> 3); }
};
template <typename V, int N> struct RowSm {
  V* buf;
  __device__ __forceinline__ void put(int g, int p, V x) const {
    buf[g * RowLayout<V, N>::LD + RowLayout<V, N>::idx(p)] = x;
  }
  __device__ __forceinline__ V get(int g, int p) const { return buf[g * RowLayout<V, N>::LD + RowLayout<V, N>::idx(p)]; }
};

template <typename T, bool INV, int N>
__global__ void __launch_bounds__(512) k_cols_ct(typename Cx<T>::t* __restrict__ planes,
                                                 const typename Cx<T>::t* __restrict__ tw, int h1, int kc,
                                                 const int* __restrict__ zr) {
  typedef typename Cx<T>::t V;
  if (zr && ((int)blockIdx.y / 6 < zr[0] || (int)blockIdx.y / 6 >= zr[1])) return;  // layer without input
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int T8 = N / 8;
  const int f = threadIdx.x % kc, t = threadIdx.x / kc;
  V* col = planes + (size_t)blockIdx.y * N * h1 + (size_t)blockIdx.x * kc + f;
  V v[1][8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[0][m] = col[(size_t)(t + m * T8) * h1];
  ColSm<V> sm{reinterpret_cast<V*>(smraw), kc, f};
  fft_ct<V, INV, N, 1, 1>(v, t, sm, tw);
#pragma unroll
  for (int m = 0; m < 8; ++m) col[(size_t)(t + m * T8) * h1] = v[0][m];
}

// FP32 column FFTs with 16-byte global accesses: a thread owns two adjacent columns (one
// float4 per row holds both), so every load and store moves 16 bytes; CW columns per CTA
// (CW = 16: every row access of a CTA is one whole 128-byte line).
// Interleaved exchange: entry p of column c at buf[p * CW + c].
template <int CW> struct ColPairSm {
  float2* buf;
  int f2;  // column pair
  __device__ __forceinline__ void put(int g, int p, float2 x) const { buf[p * CW + 2 * f2 + g] = x; }
  __device__ __forceinline__ float2 get(int g, int p) const { return buf[p * CW + 2 * f2 + g]; }
};

template <int N, int CW> struct ColsV {
  static constexpr int threads = N / 16 * CW;
  static constexpr int min_blocks = CW == 16 ? 1024 / threads : 1;  // CW = 16: 64 registers
};

// one CW-column block of one plane: tid in [0, N / 16 * CW), sm the block's [N][CW] exchange
// area; a group that has no block (live false) takes part in the exchange barriers only
template <bool INV, int N, int CW>
__device__ __forceinline__ void cols_v_body(float2* __restrict__ planes, const float2* __restrict__ tw, int h1,
                                            size_t plane, int cblk, int tid, float2* sm, bool live) {
  constexpr int T8 = N / 8, NP = CW / 2;
  const int f2 = tid % NP, t = tid / NP;
  float4* col = reinterpret_cast<float4*>(planes + plane * N * h1 + (size_t)cblk * CW + 2 * f2);
  const size_t rs = (size_t)h1 / 2;  // row stride in float4
  float2 v[2][8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const float4 a = live ? col[(size_t)(t + m * T8) * rs] : make_float4(0.f, 0.f, 0.f, 0.f);
    v[0][m] = make_float2(a.x, a.y);
    v[1][m] = make_float2(a.z, a.w);
  }
  ColPairSm<CW> x{sm, f2};
  fft_ct<float2, INV, N, 2, 1>(v, t, x, tw);
  if (live) {
#pragma unroll
    for (int m = 0; m < 8; ++m)
      col[(size_t)(t + m * T8) * rs] = make_float4(v[0][m].x, v[0][m].y, v[1][m].x, v[1][m].y);
  }
}

template <bool INV, int N, int CW>
__global__ void __launch_bounds__(ColsV<N, CW>::threads, ColsV<N, CW>::min_blocks)
    k_cols_v(float2* __restrict__ planes, const float2* __restrict__ tw, int h1, const int* __restrict__ zr) {
  if (zr && ((int)blockIdx.y / 6 < zr[0] || (int)blockIdx.y / 6 >= zr[1])) return;  // layer without input
  extern __shared__ __align__(16) unsigned char smraw[];
  cols_v_body<INV, N, CW>(planes, tw, h1, blockIdx.y, blockIdx.x, threadIdx.x, reinterpret_cast<float2*>(smraw), true);
}

// Surface displacement of a pressure, column pass fused: forward FFT along x2 of kc k1
// columns, multiplication by the surface compliance u3_hat = (1 - nu) / (mu q) p_hat (zero on
// mode 0 and on the Nyquist row k2 = N2/2, as the Boussinesq kernel), inverse FFT, in one
// kernel (a column is whole inside the CTA).  The row passes stay separate.
template <typename T, int N>
__global__ void __launch_bounds__(512) k_cols_conv(typename Cx<T>::t* __restrict__ plane,
                                                   const typename Cx<T>::t* __restrict__ tw, int h1, int kc, T w1,
                                                   T w2, T nu, T mu) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int T8 = N / 8;
  const int f = threadIdx.x % kc, t = threadIdx.x / kc;
  const int k1 = blockIdx.x * kc + f;
  V* col = plane + k1;
  V v[1][8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[0][m] = col[(size_t)(t + m * T8) * h1];
  ColSm<V> sm{reinterpret_cast<V*>(smraw), kc, f};
  fft_ct<V, false, N, 1, 1>(v, t, sm, tw);
  const T q1 = w1 * (T)k1;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int k2 = t + m * T8;
    const int k2s = k2 < N / 2 ? k2 : k2 - N;
    const T q2 = w2 * (T)k2s;
    const T q = sqrt(q1 * q1 + q2 * q2);
    const bool none = (k1 == 0 && k2 == 0) || k2 == N / 2;
    v[0][m] = none ? mk<V>(0, 0) : cscale(v[0][m], ((T)1 - nu) / (mu * q));
  }
  __syncthreads();  // the exchange area is reused by the inverse transform
  fft_ct<V, true, N, 1, 1>(v, t, sm, tw);
#pragma unroll
  for (int m = 0; m < 8; ++m) col[(size_t)(t + m * T8) * h1] = v[0][m];
}

template <typename V>
__device__ __forceinline__ void split_pair_ct(V zk, V zmk, V& A, V& B) {
  typedef decltype(V::x) T;
  const V c = cconj(zmk);
  const V s = cadd(zk, c), d = csub(zk, c);
  A = cscale(s, (T)0.5);
  B = mk<V>((T)0.5 * d.y, (T)-0.5 * d.x);
}

template <typename T, int N>
__global__ void __launch_bounds__(256) k_rows_fwd6_ct(const T* __restrict__ eps_p, typename Cx<T>::t* __restrict__ spec,
                                                      T* __restrict__ nq, const typename Cx<T>::t* __restrict__ tw,
                                                      int n2, int rb, int z0, T lam, T mu, const int* __restrict__ zr) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int T8 = N / 8, LD = RowLayout<V, N>::LD, H1 = N / 2;
  const int r = threadIdx.x / T8, t = threadIdx.x % T8;
  const int z = z0 + blockIdx.y;
  if (zr && (z < zr[0] || z >= zr[1])) return;  // layer without input
  const int x2 = blockIdx.x * rb + r;
  V v[3][8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int x1 = t + m * T8;
    T e[6], w[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = eps_p[(((size_t)z * 6 + c) * n2 + x2) * N + x1];
    hooke6_ct(e, w, lam, mu);
    v[0][m] = mk<V>(w[0], w[1]);
    v[1][m] = mk<V>(w[2], w[3]);
    v[2][m] = mk<V>(w[4], w[5]);
  }
  RowSm<V, N> sm{reinterpret_cast<V*>(smraw) + (size_t)r * 3 * LD};
  fft_ct<V, false, N, 3, 1>(v, t, sm, tw);
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int m = 0; m < 8; ++m) sm.put(g, t + m * T8, v[g][m]);
  __syncthreads();
  for (int idx = t; idx < 3 * (H1 + 1); idx += T8) {
    const int g = idx / (H1 + 1), k = idx - g * (H1 + 1);
    V A, B;
    split_pair_ct(sm.get(g, k), sm.get(g, (N - k) & (N - 1)), A, B);
    const int ca = 2 * g, cb = 2 * g + 1;
    if (k < H1) {
      spec[(((size_t)z * 6 + ca) * n2 + x2) * H1 + k] = A;
      spec[(((size_t)z * 6 + cb) * n2 + x2) * H1 + k] = B;
    } else {
      nq[((size_t)z * 6 + ca) * n2 + x2] = A.x;
      nq[((size_t)z * 6 + cb) * n2 + x2] = B.x;
    }
  }
}

// inverse row FFTs of row x2 of layer z (thread t of the row's N / 8; sm the row's exchange
// area [3][LD])
template <typename T, int N>
__device__ __forceinline__ void rows_inv6_body(const typename Cx<T>::t* __restrict__ spec, const T* __restrict__ nq,
                                               T* __restrict__ out, const typename Cx<T>::t* __restrict__ tw, int n2,
                                               int z, int x2, int t, typename Cx<T>::t* smrow, T nq_scale, T scale) {
  typedef typename Cx<T>::t V;
  constexpr int T8 = N / 8, H1 = N / 2;
  V v[3][8];
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const int ca = 2 * g, cb = 2 * g + 1;
    const V* sa = spec + (((size_t)z * 6 + ca) * n2 + x2) * H1;
    const V* sb = spec + (((size_t)z * 6 + cb) * n2 + x2) * H1;
    V ra[8], rbv[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = t + m * T8;
      const int kk = k < H1 ? k : (k > H1 ? N - k : 0);
      ra[m] = sa[kk];
      rbv[m] = sb[kk];
    }
    const T na = nq_scale == (T)0 ? (T)0 : nq_scale * nq[((size_t)z * 6 + ca) * n2 + x2];
    const T nb = nq_scale == (T)0 ? (T)0 : nq_scale * nq[((size_t)z * 6 + cb) * n2 + x2];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = t + m * T8;
      V A = ra[m], B = rbv[m];
      if (k > H1) { A = cconj(A); B = cconj(B); }
      if (k == H1) { A = mk<V>(na, 0); B = mk<V>(nb, 0); }
      v[g][m] = cadd(A, cmuli(B));
    }
  }
  RowSm<V, N> sm{smrow};
  fft_ct<V, true, N, 3, 1>(v, t, sm, tw);
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int x1 = t + m * T8;
      out[(((size_t)z * 6 + 2 * g) * n2 + x2) * N + x1] = v[g][m].x * scale;
      out[(((size_t)z * 6 + 2 * g + 1) * n2 + x2) * N + x1] = v[g][m].y * scale;
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(256) k_rows_inv6_ct(const typename Cx<T>::t* __restrict__ spec,
                                                      const T* __restrict__ nq, T* __restrict__ out,
                                                      const typename Cx<T>::t* __restrict__ tw, int n2, int rb, int z0,
                                                      T nq_scale, T scale) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int T8 = N / 8, LD = RowLayout<V, N>::LD;
  const int r = threadIdx.x / T8, t = threadIdx.x % T8;
  rows_inv6_body<T, N>(spec, nq, out, tw, n2, z0 + blockIdx.y, blockIdx.x * rb + r, t,
                       reinterpret_cast<V*>(smraw) + (size_t)r * 3 * LD, nq_scale, scale);
}

// FP32 forward row pass with 16-byte global accesses: the CTA's six eps_p rows are staged in
// shared memory with 16-byte cp.async copies and read from there in the FFT's strided order;
// the staging area then serves as the FFT exchange area, and the half spectrum leaves as
// float4 pairs of entries.  (Staging the inverse pass the same way made it slower: 0.254
// against 0.183 ms at 512 x 512 x 64, from the extra shared-memory traffic and registers.)
// row stride (floats) of the forward rows' staging area: rows of 64 or 128 points put two or
// four rows in one warp, which would read the same banks; N / 8 extra floats shift each row
// by a warp's span of one row
template <int N> struct StageLd {
  static constexpr int v = N <= 128 ? N + N / 8 : N;
};

// forward row FFTs of rows x2b .. x2b + rb - 1 of layer z by the CTA's rb * N / 8 threads;
// smraw the CTA's staging and exchange area
template <int N>
__device__ __forceinline__ void rows_fwd6_v_body(const float* __restrict__ eps_p, float2* __restrict__ spec,
                                                 float* __restrict__ nq, const float2* __restrict__ tw, int n2, int rb,
                                                 int z, int x2b, float lam, float mu, unsigned char* smraw) {
  constexpr int T8 = N / 8, LD = RowLayout<float2, N>::LD, H1 = N / 2;
  constexpr int SLD = StageLd<N>::v;
  const int r = threadIdx.x / T8, t = threadIdx.x % T8;
  const int x2 = x2b + r;
  float* stg = reinterpret_cast<float*>(smraw);  // [6][rb][SLD]
  const int per_c = rb * N / 4;
  for (int i = threadIdx.x; i < 6 * per_c; i += blockDim.x) {
    const int c = i / per_c, j = i - c * per_c;
    float* dst = stg + (size_t)c * rb * SLD + 4 * j;
    if constexpr (SLD != N) {
      const int row = (4 * j) / N;
      dst += row * (SLD - N);
    }
    cp_async_16(dst, eps_p + (((size_t)z * 6 + c) * n2 + x2b) * N + 4 * j);
  }
  cp_async_wait_all();
  __syncthreads();
  float2 v[3][8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int x1 = t + m * T8;
    float e[6], w[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = stg[((size_t)c * rb + r) * SLD + x1];
    hooke6_ct(e, w, lam, mu);
    v[0][m] = make_float2(w[0], w[1]);
    v[1][m] = make_float2(w[2], w[3]);
    v[2][m] = make_float2(w[4], w[5]);
  }
  __syncthreads();  // staging is dead: the exchange area takes its place
  RowSm<float2, N> sm{reinterpret_cast<float2*>(smraw) + (size_t)r * 3 * LD};
  fft_ct<float2, false, N, 3, 1>(v, t, sm, tw);
#pragma unroll
  for (int g = 0; g < 3; ++g)
#pragma unroll
    for (int m = 0; m < 8; ++m) sm.put(g, t + m * T8, v[g][m]);
  __syncthreads();
  for (int idx = t; idx < 3 * (H1 / 2); idx += T8) {
    const int g = idx / (H1 / 2), k = 2 * (idx - g * (H1 / 2));
    float2 A0, B0, A1, B1;
    split_pair_ct(sm.get(g, k), sm.get(g, (N - k) & (N - 1)), A0, B0);
    split_pair_ct(sm.get(g, k + 1), sm.get(g, N - k - 1), A1, B1);
    float4* ra = reinterpret_cast<float4*>(spec + (((size_t)z * 6 + 2 * g) * n2 + x2) * H1 + k);
    float4* rbp = reinterpret_cast<float4*>(spec + (((size_t)z * 6 + 2 * g + 1) * n2 + x2) * H1 + k);
    *ra = make_float4(A0.x, A0.y, A1.x, A1.y);
    *rbp = make_float4(B0.x, B0.y, B1.x, B1.y);
  }
  if (t < 3) {
    float2 A, B;
    split_pair_ct(sm.get(t, H1), sm.get(t, H1), A, B);
    nq[((size_t)z * 6 + 2 * t) * n2 + x2] = A.x;
    nq[((size_t)z * 6 + 2 * t + 1) * n2 + x2] = B.x;
  }
}

template <int N>
__global__ void __launch_bounds__(256) k_rows_fwd6_v(const float* __restrict__ eps_p, float2* __restrict__ spec,
                                                     float* __restrict__ nq, const float2* __restrict__ tw, int n2,
                                                     int rb, int z0, float lam, float mu, const int* __restrict__ zr) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int z = z0 + blockIdx.y;
  if (zr && (z < zr[0] || z >= zr[1])) return;  // layer without input
  rows_fwd6_v_body<N>(eps_p, spec, nq, tw, n2, rb, z, blockIdx.x * rb, lam, mu, smraw);
}

template <typename K> void smem_attr(K kern, size_t smem) {
  smem_cap(kern);
}

inline int ct_rows(int n1, int n2) {
  int rb = 256 / (n1 >> 3);
  if (rb > 8) rb = 8;
  while (rb > n2) rb >>= 1;
  return rb;
}

template <int N, int CW> void cols_v_launch(const fvim_ctx* c, bool inverse, void* planes, int nplanes, const int* zr) {
  dim3 grid(c->h1 / CW, nplanes);
  const size_t sm = (size_t)N * CW * sizeof(float2);
  if (inverse) {
    smem_attr(k_cols_v<true, N, CW>, sm);
    k_cols_v<true, N, CW><<<grid, ColsV<N, CW>::threads, sm, c->stream>>>((float2*)planes, (const float2*)c->tw2,
                                                                          c->h1, zr);
  } else {
    smem_attr(k_cols_v<false, N, CW>, sm);
    k_cols_v<false, N, CW><<<grid, ColsV<N, CW>::threads, sm, c->stream>>>((float2*)planes, (const float2*)c->tw2,
                                                                           c->h1, zr);
  }
}

template <typename T, int N> void cols_n(const fvim_ctx* c, bool inverse, void* planes, int nplanes, const int* zr) {
  typedef typename Cx<T>::t V;
  if constexpr (sizeof(T) == 4 && N >= 64) {
    // 16 columns per CTA (whole 128-byte rows): N threads, 1024 at N = 1024 (one CTA per SM)
    if (c->h1 % 16 == 0) {
      cols_v_launch<N, 16>(c, inverse, planes, nplanes, zr);
      return;
    }
    if (c->h1 % 8 == 0) {
      cols_v_launch<N, 8>(c, inverse, planes, nplanes, zr);
      return;
    }
  }
  int kc = (int)(128 / sizeof(V));  // 128-byte rows
  while (kc > 1 && kc * (N / 8) > 512) kc >>= 1;
  if (kc > c->h1) kc = c->h1;
  const int threads = kc * (N / 8);
  const size_t smem = (size_t)kc * N * sizeof(V);
  dim3 grid(c->h1 / kc, nplanes);
  if (inverse) {
    smem_attr(k_cols_ct<T, true, N>, smem);
    k_cols_ct<T, true, N><<<grid, threads, smem, c->stream>>>((V*)planes, (const V*)c->tw2, c->h1, kc, zr);
  } else {
    smem_attr(k_cols_ct<T, false, N>, smem);
    k_cols_ct<T, false, N><<<grid, threads, smem, c->stream>>>((V*)planes, (const V*)c->tw2, c->h1, kc, zr);
  }
}

template <typename T, int N> void rows_fwd_n(const fvim_ctx* c, const T* eps_p, int z0, int nzs, const int* zr) {
  typedef typename Cx<T>::t V;
  const int rb = ct_rows(N, c->n2);
  if constexpr (sizeof(T) == 4 && N >= 64) {
    const size_t sm = std::max((size_t)rb * 3 * RowLayout<V, N>::LD * sizeof(V), (size_t)6 * rb * StageLd<N>::v * sizeof(T));
    dim3 grid(c->n2 / rb, nzs);
    smem_attr(k_rows_fwd6_v<N>, sm);
    k_rows_fwd6_v<N><<<grid, rb * (N / 8), sm, c->stream>>>((const float*)eps_p, (float2*)c->spec, (float*)c->nq,
                                                            (const float2*)c->tw1, c->n2, rb, z0, (float)c->lam,
                                                            (float)c->mu, zr);
    return;
  }
  const size_t smem = (size_t)rb * 3 * RowLayout<V, N>::LD * sizeof(V);
  dim3 grid(c->n2 / rb, nzs);
  smem_attr(k_rows_fwd6_ct<T, N>, smem);
  k_rows_fwd6_ct<T, N><<<grid, rb * (N / 8), smem, c->stream>>>(eps_p, (V*)c->spec, (T*)c->nq, (const V*)c->tw1,
                                                              c->n2, rb, z0, (T)c->lam, (T)c->mu, zr);
}

template <typename T, int N> void rows_inv_n(const fvim_ctx* c, T* out, T nq_scale, int z0, int nzs) {
  typedef typename Cx<T>::t V;
  int rb = ct_rows(N, c->n2);
  // smaller CTAs in FP32 (128 threads at N = 512 and 1024): 5 instead of 2 per SM at ~100 registers
  if (sizeof(T) == 4 && (rb >= 4 || N >= 1024)) rb = std::max(1, rb / 2);
  const size_t smem = (size_t)rb * 3 * RowLayout<V, N>::LD * sizeof(V);
  dim3 grid(c->n2 / rb, nzs);
  const T scale = (T)(1.0 / ((double)N * (double)c->n2));
  smem_attr(k_rows_inv6_ct<T, N>, smem);
  k_rows_inv6_ct<T, N><<<grid, rb * (N / 8), smem, c->stream>>>((const V*)c->spec, (const T*)c->nq, out,
                                                              (const V*)c->tw1, c->n2, rb, z0, nq_scale, scale);
}

// ---- grouped launches: every problem of a GrpTable in one launch per pass ---------------
// A CTA finds its problem by the table's CTA offsets and runs the same body as the
// single-problem kernels, so each problem's results are those of its own launch sequence.
// Shapes are chosen so that every N in 64..512 fills the same CTA: forward rows 2048 / N1 rows
// per CTA (256 threads), inverse rows 1024 / N1 rows (128 threads), columns 512 / N2 blocks of
// 16 columns (512 threads, N2 threads per block).
constexpr int kGrpRowsFwdSmem = 2048 * 3 * 9 / 8 * 8;    // = 6 * 2048 * 9 / 8 * 4 bytes of staging
constexpr int kGrpRowsInvSmem = 1024 * 3 * 9 / 8 * 8;
constexpr int kGrpColsSmem = 512 * 16 * 8;

template <int N> __device__ __forceinline__ void grp_rows_fwd_case(const GrpProb& P, int local, unsigned char* sm) {
  const int rb = 2048 / N, nrb = P.n2 / rb;
  const int z = local / nrb, x2b = (local - z * nrb) * rb;
  rows_fwd6_v_body<N>(P.eps, P.spec, P.nq, P.tw1, P.n2, rb, z, x2b, P.lam, P.mu, sm);
}

__global__ void __launch_bounds__(256) k_grp_rows_fwd(const __grid_constant__ GrpTable tab) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pi = grp_find(tab, blockIdx.x);
  const GrpProb& P = tab.p[pi];
  const int local = (int)blockIdx.x - tab.start[pi];
  switch (P.n1) {
    case 64: grp_rows_fwd_case<64>(P, local, smraw); break;
    case 128: grp_rows_fwd_case<128>(P, local, smraw); break;
    case 256: grp_rows_fwd_case<256>(P, local, smraw); break;
    case 512: grp_rows_fwd_case<512>(P, local, smraw); break;
    default: break;
  }
}

template <int N> __device__ __forceinline__ void grp_rows_inv_case(const GrpProb& P, int local, unsigned char* sm) {
  constexpr int T8 = N / 8, LD = RowLayout<float2, N>::LD;
  const int rb = 1024 / N, nrb = P.n2 / rb;
  const int z = local / nrb, r = threadIdx.x / T8, t = threadIdx.x % T8;
  const int x2 = (local - z * nrb) * rb + r;
  rows_inv6_body<float, N>(P.spec, P.nq, P.out, P.tw1, P.n2, z, x2, t,
                           reinterpret_cast<float2*>(sm) + (size_t)r * 3 * LD, P.nq_scale, P.scale);
}

__global__ void __launch_bounds__(128) k_grp_rows_inv(const __grid_constant__ GrpTable tab) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pi = grp_find(tab, blockIdx.x);
  const GrpProb& P = tab.p[pi];
  const int local = (int)blockIdx.x - tab.start[pi];
  switch (P.n1) {
    case 64: grp_rows_inv_case<64>(P, local, smraw); break;
    case 128: grp_rows_inv_case<128>(P, local, smraw); break;
    case 256: grp_rows_inv_case<256>(P, local, smraw); break;
    case 512: grp_rows_inv_case<512>(P, local, smraw); break;
    default: break;
  }
}

template <bool INV, int N>
__device__ __forceinline__ void grp_cols_case(const GrpProb& P, int local, unsigned char* sm) {
  constexpr int G = 512 / N;  // column blocks per CTA, N threads each
  const int g = threadIdx.x / N, tid = threadIdx.x - g * N;
  const int ncb = P.h1 / 16, items = P.nz * 6 * ncb;
  const int item = local * G + g;
  const bool live = item < items;
  const int plane = live ? item / ncb : 0, cblk = live ? item - plane * ncb : 0;
  cols_v_body<INV, N, 16>(P.spec, P.tw2, P.h1, (size_t)plane, cblk, tid,
                          reinterpret_cast<float2*>(sm) + (size_t)g * N * 16, live);
}

template <bool INV> __global__ void __launch_bounds__(512, 2) k_grp_cols(const __grid_constant__ GrpTable tab) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int pi = grp_find(tab, blockIdx.x);
  const GrpProb& P = tab.p[pi];
  const int local = (int)blockIdx.x - tab.start[pi];
  switch (P.n2) {
    case 64: grp_cols_case<INV, 64>(P, local, smraw); break;
    case 128: grp_cols_case<INV, 128>(P, local, smraw); break;
    case 256: grp_cols_case<INV, 256>(P, local, smraw); break;
    case 512: grp_cols_case<INV, 512>(P, local, smraw); break;
    default: break;
  }
}

}  // namespace

#define FVIM_CT_SIZES(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024)

template <typename T> bool launch_cols_ct(const fvim_ctx* c, bool inverse, void* planes, int nplanes, const int* zr) {
#define CASE(N)                                 \
  if (c->n2 == N) {                             \
    cols_n<T, N>(c, inverse, planes, nplanes, zr); \
    return true;                                \
  }
  FVIM_CT_SIZES(CASE)
#undef CASE
  return false;
}

template <typename T, int N> void cols_conv_n(const fvim_ctx* c) {
  typedef typename Cx<T>::t V;
  int kc = (int)(128 / sizeof(V));  // 128-byte rows
  while (kc > 1 && kc * (N / 8) > 512) kc >>= 1;
  if (kc > c->h1) kc = c->h1;
  const size_t smem = (size_t)kc * N * sizeof(V);
  smem_attr(k_cols_conv<T, N>, smem);
  const double two_pi = 6.283185307179586476925;
  k_cols_conv<T, N><<<c->h1 / kc, kc * (N / 8), smem, c->stream>>>(
      (V*)c->surf, (const V*)c->tw2, c->h1, kc, (T)(two_pi / c->L1), (T)(two_pi / c->L2), (T)c->nu, (T)c->mu);
}

template <typename T> bool launch_cols_conv_ct(const fvim_ctx* c) {
#define CASE(N)              \
  if (c->n2 == N) {          \
    cols_conv_n<T, N>(c);    \
    return true;             \
  }
  FVIM_CT_SIZES(CASE)
#undef CASE
  return false;
}

template <typename T> bool launch_rows_fwd6_ct(const fvim_ctx* c, const T* eps_p, int z0, int nzs, const int* zr) {
#define CASE(N)                              \
  if (c->n1 == N) {                          \
    rows_fwd_n<T, N>(c, eps_p, z0, nzs, zr); \
    return true;                             \
  }
  FVIM_CT_SIZES(CASE)
#undef CASE
  return false;
}

template <typename T> bool launch_rows_inv6_ct(const fvim_ctx* c, T* out, T nq_scale, int z0, int nzs) {
#define CASE(N)                                     \
  if (c->n1 == N) {                                 \
    rows_inv_n<T, N>(c, out, nq_scale, z0, nzs);    \
    return true;                                    \
  }
  FVIM_CT_SIZES(CASE)
#undef CASE
  return false;
}

template bool launch_cols_ct<float>(const fvim_ctx*, bool, void*, int, const int*);
template bool launch_cols_conv_ct<float>(const fvim_ctx*);
template bool launch_cols_conv_ct<double>(const fvim_ctx*);
template bool launch_cols_ct<double>(const fvim_ctx*, bool, void*, int, const int*);
template bool launch_rows_fwd6_ct<float>(const fvim_ctx*, const float*, int, int, const int*);
template bool launch_rows_fwd6_ct<double>(const fvim_ctx*, const double*, int, int, const int*);
template bool launch_rows_inv6_ct<float>(const fvim_ctx*, float*, float, int, int);
template bool launch_rows_inv6_ct<double>(const fvim_ctx*, double*, double, int, int);

int launch_grp_rows_fwd(GrpTable& t, cudaStream_t s) {
  int b = 0;
  for (int i = 0; i < t.n; ++i) {
    t.start[i] = b;
    b += t.p[i].nz * (t.p[i].n2 / (2048 / t.p[i].n1));
  }
  t.start[t.n] = b;
  if (b == 0) return FVIM_OK;
  smem_attr(k_grp_rows_fwd, kGrpRowsFwdSmem);
  k_grp_rows_fwd<<<b, 256, kGrpRowsFwdSmem, s>>>(t);
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

int launch_grp_rows_inv(GrpTable& t, cudaStream_t s) {
  int b = 0;
  for (int i = 0; i < t.n; ++i) {
    t.start[i] = b;
    b += t.p[i].nz * (t.p[i].n2 / (1024 / t.p[i].n1));
  }
  t.start[t.n] = b;
  if (b == 0) return FVIM_OK;
  smem_attr(k_grp_rows_inv, kGrpRowsInvSmem);
  k_grp_rows_inv<<<b, 128, kGrpRowsInvSmem, s>>>(t);
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

int launch_grp_cols(GrpTable& t, bool inverse, cudaStream_t s) {
  int b = 0;
  for (int i = 0; i < t.n; ++i) {
    t.start[i] = b;
    const int items = t.p[i].nz * 6 * (t.p[i].h1 / 16), per = 512 / t.p[i].n2;
    b += (items + per - 1) / per;
  }
  t.start[t.n] = b;
  if (b == 0) return FVIM_OK;
  if (inverse) {
    smem_attr(k_grp_cols<true>, kGrpColsSmem);
    k_grp_cols<true><<<b, 512, kGrpColsSmem, s>>>(t);
  } else {
    smem_attr(k_grp_cols<false>, kGrpColsSmem);
    k_grp_cols<false><<<b, 512, kGrpColsSmem, s>>>(t);
  }
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

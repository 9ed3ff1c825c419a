// In-plane transforms of the volume and surface fields (Sec. 3.1, Eq. dft: the DFT of
// the nodal values of every layer, unnormalised forward, 1/(N1 N2) on the way back).
//
// Layout of the half spectrum kept between kernels (complex T):
//   spec[z][c][k2][k1], k1 in [0, N1/2)   (k1 = N1/2 is not in Z^2_N, Sec. 3.1)
//   nq[z][c][x2]         the k1 = N1/2 row coefficient (real), kept so that the stress
//                        output can return sigma_hat = -w_hat on that column.
// Rows: two real rows share one complex FFT of length N1 (z = a + i b); the halves are
// separated with the Hermitian symmetry of real data.
#include "fvim_internal.cuh"

namespace {

// threads per CTA cap: 128 registers per thread in FP32, 255 in FP64
template <typename T> struct MaxT { static constexpr int v = sizeof(T) == 4 ? 512 : 256; };

// w = C:eps_p for one voxel, six stored components (Sec. 4.2: the operator acts on C:eps_p)
template <typename T>
__device__ __forceinline__ void hooke6(const T* e, T* w, T lam, T mu) {
  const T tr = e[0] + e[1] + e[2];
  w[0] = lam * tr + 2 * mu * e[0];
  w[1] = lam * tr + 2 * mu * e[1];
  w[2] = lam * tr + 2 * mu * e[2];
  w[3] = 2 * mu * e[3];
  w[4] = 2 * mu * e[4];
  w[5] = 2 * mu * e[5];
}

// Separate the transforms A, B of two real sequences from Z = FFT(a + i b) at index k.
template <typename V>
__device__ __forceinline__ void split_pair(V zk, V zmk, V& A, V& B) {
  typedef decltype(V::x) T;
  // A = (Z(k) + conj Z(-k)) / 2 ; B = (Z(k) - conj Z(-k)) / (2 i)
  V c = cconj(zmk);
  V s = cadd(zk, c), d = csub(zk, c);
  A = cscale(s, (T)0.5);
  B = mk<V>((T)0.5 * d.y, (T)-0.5 * d.x);
}

// --- forward rows, six components with the Hooke prologue -----------------------
// grid: (N2 / RB, nzs); block: threads; each CTA handles RB rows of one layer.
template <typename T, int RB, int MAXI>
__global__ void __launch_bounds__(MaxT<T>::v) k_rows_fwd6(const T* __restrict__ eps_p, typename Cx<T>::t* __restrict__ spec,
                            T* __restrict__ nq, const typename Cx<T>::t* __restrict__ tw, int n1, int n2,
                            int z0, T lam, T mu) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* buf = reinterpret_cast<V*>(smraw);  // [RB][3][n1]
  const int z = z0 + blockIdx.y;
  const int x2b = blockIdx.x * RB;
  const int h1 = n1 >> 1;
  // load + Hooke: thread handles (row, x1)
  for (int idx = threadIdx.x; idx < RB * n1; idx += blockDim.x) {
    const int r = idx / n1, x1 = idx - r * n1;
    const int x2 = x2b + r;
    T e[6], w[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = eps_p[(((size_t)z * 6 + c) * n2 + x2) * n1 + x1];
    hooke6(e, w, lam, mu);
    V* row = buf + (size_t)r * 3 * n1;
    row[x1] = mk<V>(w[0], w[1]);
    row[n1 + x1] = mk<V>(w[2], w[3]);
    row[2 * n1 + x1] = mk<V>(w[4], w[5]);
  }
  __syncthreads();
  block_fft<V, false, MAXI>(buf, n1, 3 * RB, n1, tw);
  // unpack: k1 in [0, h1] for each pair
  for (int idx = threadIdx.x; idx < RB * 3 * (h1 + 1); idx += blockDim.x) {
    const int r = idx / (3 * (h1 + 1));
    const int rem = idx - r * 3 * (h1 + 1);
    const int p = rem / (h1 + 1), k = rem - p * (h1 + 1);
    const V* row = buf + ((size_t)r * 3 + p) * n1;
    V A, B;
    split_pair(row[k], row[(n1 - k) & (n1 - 1)], A, B);
    const int x2 = x2b + r;
    const int ca = 2 * p, cb = 2 * p + 1;
    if (k < h1) {
      spec[(((size_t)z * 6 + ca) * n2 + x2) * h1 + k] = A;
      spec[(((size_t)z * 6 + cb) * n2 + x2) * h1 + k] = B;
    } else {
      nq[((size_t)z * 6 + ca) * n2 + x2] = A.x;
      nq[((size_t)z * 6 + cb) * n2 + x2] = B.x;
    }
  }
}

// --- forward rows of a single real surface field (two rows per complex FFT) ------
template <typename T, int MAXI>
__global__ void __launch_bounds__(MaxT<T>::v) k_rows_fwd1(const T* __restrict__ f, typename Cx<T>::t* __restrict__ spec, T* __restrict__ nq,
                            const typename Cx<T>::t* __restrict__ tw, int n1, int n2) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* buf = reinterpret_cast<V*>(smraw);  // [n1]
  const int x2 = 2 * blockIdx.x;
  const int h1 = n1 >> 1;
  for (int x1 = threadIdx.x; x1 < n1; x1 += blockDim.x)
    buf[x1] = mk<V>(f[(size_t)x2 * n1 + x1], f[(size_t)(x2 + 1) * n1 + x1]);
  __syncthreads();
  block_fft<V, false, MAXI>(buf, n1, 1, n1, tw);
  for (int k = threadIdx.x; k <= h1; k += blockDim.x) {
    V A, B;
    split_pair(buf[k], buf[(n1 - k) & (n1 - 1)], A, B);
    if (k < h1) {
      spec[(size_t)x2 * h1 + k] = A;
      spec[(size_t)(x2 + 1) * h1 + k] = B;
    } else {
      nq[x2] = A.x;
      nq[x2 + 1] = B.x;
    }
  }
}

// --- columns: FFT along x2 of KC consecutive k1 columns of one plane --------------
template <typename T, bool INV, int MAXI>
__global__ void __launch_bounds__(MaxT<T>::v) k_cols(typename Cx<T>::t* __restrict__ planes, const typename Cx<T>::t* __restrict__ tw, int n2,
                       int h1, int kc) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* buf = reinterpret_cast<V*>(smraw);  // [kc][n2 + 1]
  const int ld = n2 + 1;
  V* plane = planes + (size_t)blockIdx.y * n2 * h1;
  const int k1b = blockIdx.x * kc;
  for (int idx = threadIdx.x; idx < kc * n2; idx += blockDim.x) {
    const int k2 = idx / kc, c = idx - k2 * kc;
    buf[c * ld + k2] = plane[(size_t)k2 * h1 + k1b + c];
  }
  __syncthreads();
  block_fft<V, INV, MAXI>(buf, n2, kc, ld, tw);
  for (int idx = threadIdx.x; idx < kc * n2; idx += blockDim.x) {
    const int k2 = idx / kc, c = idx - k2 * kc;
    plane[(size_t)k2 * h1 + k1b + c] = buf[c * ld + k2];
  }
}

// --- inverse rows, six components ------------------------------------------------
// nq_scale multiplies the stored k1 = N1/2 coefficient (-N2 for the stress output of the
// Mindlin operator, sigma_hat = -w_hat there; 0 when the operator has no Nyquist term).
// scale = 1/(N1 N2).
template <typename T, int RB, int MAXI>
__global__ void __launch_bounds__(MaxT<T>::v) k_rows_inv6(const typename Cx<T>::t* __restrict__ spec, const T* __restrict__ nq, T* __restrict__ out,
                            const typename Cx<T>::t* __restrict__ tw, int n1, int n2, int z0, T nq_scale, T scale) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* buf = reinterpret_cast<V*>(smraw);  // [RB][3][n1]
  const int z = z0 + blockIdx.y;
  const int x2b = blockIdx.x * RB;
  const int h1 = n1 >> 1;
  // build Z(k) = A(k) + i B(k) over the full length with A(-k) = conj A(k)
  for (int idx = threadIdx.x; idx < RB * 3 * n1; idx += blockDim.x) {
    const int r = idx / (3 * n1);
    const int rem = idx - r * 3 * n1;
    const int p = rem / n1, k = rem - p * n1;
    const int x2 = x2b + r;
    const int ca = 2 * p, cb = 2 * p + 1;
    V A, B;
    if (k == h1) {
      A = mk<V>(nq_scale == (T)0 ? (T)0 : nq_scale * nq[((size_t)z * 6 + ca) * n2 + x2], 0);
      B = mk<V>(nq_scale == (T)0 ? (T)0 : nq_scale * nq[((size_t)z * 6 + cb) * n2 + x2], 0);
    } else {
      const int kk = k < h1 ? k : n1 - k;
      A = spec[(((size_t)z * 6 + ca) * n2 + x2) * h1 + kk];
      B = spec[(((size_t)z * 6 + cb) * n2 + x2) * h1 + kk];
      if (k > h1) { A = cconj(A); B = cconj(B); }
    }
    buf[((size_t)r * 3 + p) * n1 + k] = cadd(A, cmuli(B));
  }
  __syncthreads();
  block_fft<V, true, MAXI>(buf, n1, 3 * RB, n1, tw);
  for (int idx = threadIdx.x; idx < RB * n1; idx += blockDim.x) {
    const int r = idx / n1, x1 = idx - r * n1;
    const int x2 = x2b + r;
    const V* row = buf + (size_t)r * 3 * n1;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const V v = row[p * n1 + x1];
      out[(((size_t)z * 6 + 2 * p) * n2 + x2) * n1 + x1] = v.x * scale;
      out[(((size_t)z * 6 + 2 * p + 1) * n2 + x2) * n1 + x1] = v.y * scale;
    }
  }
}

// --- inverse rows of a single surface field (two rows per complex FFT) ------------
template <typename T, int MAXI>
__global__ void __launch_bounds__(MaxT<T>::v) k_rows_inv1(const typename Cx<T>::t* __restrict__ spec, const T* __restrict__ nq, T* __restrict__ f,
                            const typename Cx<T>::t* __restrict__ tw, int n1, int n2, T nq_scale, T scale) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* buf = reinterpret_cast<V*>(smraw);
  const int x2 = 2 * blockIdx.x;
  const int h1 = n1 >> 1;
  for (int k = threadIdx.x; k < n1; k += blockDim.x) {
    V A, B;
    if (k == h1) {
      A = mk<V>(nq_scale == (T)0 ? (T)0 : nq_scale * nq[x2], 0);
      B = mk<V>(nq_scale == (T)0 ? (T)0 : nq_scale * nq[x2 + 1], 0);
    } else {
      const int kk = k < h1 ? k : n1 - k;
      A = spec[(size_t)x2 * h1 + kk];
      B = spec[(size_t)(x2 + 1) * h1 + kk];
      if (k > h1) { A = cconj(A); B = cconj(B); }
    }
    buf[k] = cadd(A, cmuli(B));
  }
  __syncthreads();
  block_fft<V, true, MAXI>(buf, n1, 1, n1, tw);
  for (int x1 = threadIdx.x; x1 < n1; x1 += blockDim.x) {
    f[(size_t)x2 * n1 + x1] = buf[x1].x * scale;
    f[(size_t)(x2 + 1) * n1 + x1] = buf[x1].y * scale;
  }
}


// ================================================================================
// Register-resident kernels (n >= 8): each thread keeps 8 strided elements of its
// transform in registers for all stages (reg_stage); shared memory is only the
// exchange between stages.  Columns keep the KC transforms of a CTA interleaved
// (128-byte rows, conflict-free); rows keep each transform contiguous with one pad
// slot every 8 entries (conflict-free Stockham scatter).
// ================================================================================
__device__ __forceinline__ int padi(int p) { return p + (p >> 3); }

// columns: CTA = KC consecutive k1 columns of one plane, KC * n2/8 threads
template <typename T, bool INV, int KC>
__global__ void __launch_bounds__(512) k_cols8(typename Cx<T>::t* __restrict__ planes,
                                                const typename Cx<T>::t* __restrict__ tw, int n2, int h1) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* buf = reinterpret_cast<V*>(smraw);  // [n2][KC]
  const int f = threadIdx.x % KC, t = threadIdx.x / KC;
  const int T8 = n2 >> 3;
  V* col = planes + (size_t)blockIdx.y * n2 * h1 + (size_t)blockIdx.x * KC + f;
  V v[8];
  int pos[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) v[m] = col[(size_t)(t + m * T8) * h1];
  int Ns = 1, rem = n2;
  bool first = true;
  while (rem > 1) {
    const int R = fft_radix(rem);
    const bool last = (rem == R);
    if (!first) {
      __syncthreads();
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = buf[(t + m * T8) * KC + f];
      if (!last) __syncthreads();
    }
    reg_stage<V, INV>(v, pos, t, n2, R, Ns, tw);
    if (!last) {
#pragma unroll
      for (int m = 0; m < 8; ++m) buf[pos[m] * KC + f] = v[m];
    }
    first = false;
    Ns *= R;
    rem /= R;
  }
#pragma unroll
  for (int m = 0; m < 8; ++m) col[(size_t)(t + m * T8) * h1] = v[m];
}

// forward rows with the Hooke prologue: CTA = RB rows of one layer, RB * n1/8 threads;
// a thread runs the three pair transforms (w11 + i w22, w33 + i w23, w13 + i w12)
template <typename T, int RB>
__global__ void __launch_bounds__(256) k_rows_fwd6_r8(const T* __restrict__ eps_p, typename Cx<T>::t* __restrict__ spec,
                                                      T* __restrict__ nq, const typename Cx<T>::t* __restrict__ tw,
                                                      int n1, int n2, int z0, T lam, T mu) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* buf = reinterpret_cast<V*>(smraw);  // [RB][3][padi(n1)]
  const int T8 = n1 >> 3;
  const int ld = n1 + T8;
  const int r = threadIdx.x / T8, t = threadIdx.x - r * T8;
  const int z = z0 + blockIdx.y;
  const int x2 = blockIdx.x * RB + r;
  const int h1 = n1 >> 1;
  V v[3][8];
  int pos[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int x1 = t + m * T8;
    T e[6], w[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) e[c] = eps_p[(((size_t)z * 6 + c) * n2 + x2) * n1 + x1];
    hooke6(e, w, lam, mu);
    v[0][m] = mk<V>(w[0], w[1]);
    v[1][m] = mk<V>(w[2], w[3]);
    v[2][m] = mk<V>(w[4], w[5]);
  }
  V* rowbuf = buf + (size_t)r * 3 * ld;
  int Ns = 1, rem = n1;
  bool first = true;
  while (rem > 1) {
    const int R = fft_radix(rem);
    if (!first) {
      __syncthreads();
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int m = 0; m < 8; ++m) v[p][m] = rowbuf[p * ld + padi(t + m * T8)];
      __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      reg_stage<V, false>(v[p], pos, t, n1, R, Ns, tw);
#pragma unroll
      for (int m = 0; m < 8; ++m) rowbuf[p * ld + padi(pos[m])] = v[p][m];
    }
    first = false;
    Ns *= R;
    rem /= R;
  }
  __syncthreads();
  // Hermitian split of the natural-order outputs: k in [0, h1]
  for (int idx = t; idx < 3 * (h1 + 1); idx += T8) {
    const int p = idx / (h1 + 1), k = idx - p * (h1 + 1);
    V A, B;
    split_pair(rowbuf[p * ld + padi(k)], rowbuf[p * ld + padi((n1 - k) & (n1 - 1))], A, B);
    const int ca = 2 * p, cb = 2 * p + 1;
    if (k < h1) {
      spec[(((size_t)z * 6 + ca) * n2 + x2) * h1 + k] = A;
      spec[(((size_t)z * 6 + cb) * n2 + x2) * h1 + k] = B;
    } else {
      nq[((size_t)z * 6 + ca) * n2 + x2] = A.x;
      nq[((size_t)z * 6 + cb) * n2 + x2] = B.x;
    }
  }
}

// inverse rows: Hermitian rebuild straight from the half spectrum into registers,
// inverse transforms, scaled real/imaginary parts stored per component
template <typename T, int RB>
__global__ void __launch_bounds__(256) k_rows_inv6_r8(const typename Cx<T>::t* __restrict__ spec,
                                                      const T* __restrict__ nq, T* __restrict__ out,
                                                      const typename Cx<T>::t* __restrict__ tw, int n1, int n2, int z0,
                                                      T nq_scale, T scale) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* buf = reinterpret_cast<V*>(smraw);  // [RB][3][padi(n1)]
  const int T8 = n1 >> 3;
  const int ld = n1 + T8;
  const int r = threadIdx.x / T8, t = threadIdx.x - r * T8;
  const int z = z0 + blockIdx.y;
  const int x2 = blockIdx.x * RB + r;
  const int h1 = n1 >> 1;
  V v[3][8];
  int pos[8];
#pragma unroll
  for (int p = 0; p < 3; ++p) {
    const int ca = 2 * p, cb = 2 * p + 1;
    const V* sa = spec + (((size_t)z * 6 + ca) * n2 + x2) * h1;
    const V* sb = spec + (((size_t)z * 6 + cb) * n2 + x2) * h1;
    // unconditional loads first (all in flight), then the Hermitian selection
    V ra[8], rb[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = t + m * T8;
      const int kk = k < h1 ? k : (k > h1 ? n1 - k : 0);
      ra[m] = sa[kk];
      rb[m] = sb[kk];
    }
    const T na = nq_scale == (T)0 ? (T)0 : nq_scale * nq[((size_t)z * 6 + ca) * n2 + x2];
    const T nb = nq_scale == (T)0 ? (T)0 : nq_scale * nq[((size_t)z * 6 + cb) * n2 + x2];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int k = t + m * T8;
      V A = ra[m], B = rb[m];
      if (k > h1) { A = cconj(A); B = cconj(B); }
      if (k == h1) { A = mk<V>(na, 0); B = mk<V>(nb, 0); }
      v[p][m] = cadd(A, cmuli(B));
    }
  }
  V* rowbuf = buf + (size_t)r * 3 * ld;
  int Ns = 1, rem = n1;
  bool first = true;
  while (rem > 1) {
    const int R = fft_radix(rem);
    const bool last = (rem == R);
    if (!first) {
      __syncthreads();
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int m = 0; m < 8; ++m) v[p][m] = rowbuf[p * ld + padi(t + m * T8)];
      if (!last) __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      reg_stage<V, true>(v[p], pos, t, n1, R, Ns, tw);
      if (!last) {
#pragma unroll
        for (int m = 0; m < 8; ++m) rowbuf[p * ld + padi(pos[m])] = v[p][m];
      }
    }
    first = false;
    Ns *= R;
    rem /= R;
  }
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int x1 = t + m * T8;
      out[(((size_t)z * 6 + 2 * p) * n2 + x2) * n1 + x1] = v[p][m].x * scale;
      out[(((size_t)z * 6 + 2 * p + 1) * n2 + x2) * n1 + x1] = v[p][m].y * scale;
    }
}

inline int round_threads(int t, int cap) {
  t = (t + 31) / 32 * 32;
  if (t < 64) t = 64;
  if (t > cap) t = cap;
  return t;
}

// items per thread (MAXI) and threads for a batch of nfft transforms of length n
template <typename T> bool fft_shape(int nfft, int n, int& maxi, int& threads) {
  const int items = nfft * n / fft_rmin(n);
  const int cap = MaxT<T>::v;
  if (items <= 2 * cap) maxi = 2;
  else if (items <= 4 * cap) maxi = 4;
  else return false;
  threads = round_threads((items + maxi - 1) / maxi, cap);
  return true;
}

// rows per CTA: a few rows when they are short, within the per-thread item budget
template <typename T> int row_block(int n1, int n2) {
  int rb = n1 <= 256 ? 4 : (n1 <= 512 ? 2 : 1);
  while (rb > n2) rb >>= 1;
  while (rb > 1 && 3 * rb * n1 / fft_rmin(n1) > 2 * MaxT<T>::v) rb >>= 1;
  return rb;
}

template <typename K> void set_smem(K kern, size_t smem) {
  smem_cap(kern);
}

}  // namespace

// rows per CTA of the register-resident row kernels (256 threads, n1/8 per row)
inline int r8_rows(int n1, int n2) {
  int rb = 256 / (n1 >> 3);
  if (rb > 8) rb = 8;
  while (rb > n2) rb >>= 1;
  return rb;
}

template <typename T> int launch_rows_fwd6(const fvim_ctx* c, const T* eps_p, int z0, int nzs, const int* zr) {
  typedef typename Cx<T>::t V;
  const int n1 = c->n1, n2 = c->n2;
  if (launch_rows_fwd6_ct<T>(c, eps_p, z0, nzs, zr)) {
    FVIM_CUDA_CHECK_LAUNCH();
    return FVIM_OK;
  }
  if (n1 >= 8 && n1 <= 2048) {
    const int RB = r8_rows(n1, n2);
    const int threads = RB * (n1 >> 3);
    const size_t smem = (size_t)RB * 3 * (n1 + n1 / 8) * sizeof(V);
    dim3 grid(n2 / RB, nzs);
    const T lam = (T)c->lam, mu = (T)c->mu;
#define RF(RBV)                                                                                    \
  if (RB == RBV) {                                                                                 \
    set_smem(k_rows_fwd6_r8<T, RBV>, smem);                                                        \
    k_rows_fwd6_r8<T, RBV><<<grid, threads, smem, c->stream>>>(eps_p, (V*)c->spec, (T*)c->nq,      \
                                                               (const V*)c->tw1, n1, n2, z0, lam, mu); \
  }
    RF(8) RF(4) RF(2) RF(1)
#undef RF
    FVIM_CUDA_CHECK_LAUNCH();
    return FVIM_OK;
  }
  const int RB = row_block<T>(n1, n2);
  int maxi, threads;
  if (n2 % RB || !fft_shape<T>(3 * RB, n1, maxi, threads)) return FVIM_ERR_UNSUPPORTED;
  const size_t smem = (size_t)RB * 3 * n1 * sizeof(V);
  dim3 grid(n2 / RB, nzs);
  const T lam = (T)c->lam, mu = (T)c->mu;
  V* spec = (V*)c->spec;
  T* nq = (T*)c->nq;
  const V* tw = (const V*)c->tw1;
#define FWD6(RBV, MI)                                                                      \
  if (RB == RBV && maxi == MI) {                                                           \
    set_smem(k_rows_fwd6<T, RBV, MI>, smem);                                               \
    k_rows_fwd6<T, RBV, MI><<<grid, threads, smem, c->stream>>>(eps_p, spec, nq, tw, n1, n2, z0, lam, mu); \
  }
  FWD6(4, 2) FWD6(2, 2) FWD6(1, 2) FWD6(4, 4) FWD6(2, 4) FWD6(1, 4)
#undef FWD6
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

template <typename T> int launch_rows_fwd1(const fvim_ctx* c, const T* f) {
  typedef typename Cx<T>::t V;
  const int n1 = c->n1, n2 = c->n2;
  int maxi, threads;
  if (!fft_shape<T>(1, n1, maxi, threads)) return FVIM_ERR_UNSUPPORTED;
  const size_t smem = (size_t)n1 * sizeof(V);
  if (maxi == 2)
    k_rows_fwd1<T, 2><<<n2 / 2, threads, smem, c->stream>>>(f, (V*)c->surf, (T*)c->surf_nq, (const V*)c->tw1, n1, n2);
  else
    k_rows_fwd1<T, 4><<<n2 / 2, threads, smem, c->stream>>>(f, (V*)c->surf, (T*)c->surf_nq, (const V*)c->tw1, n1, n2);
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

template <typename T> int launch_cols(const fvim_ctx* c, bool inverse, void* planes, int nplanes, const int* zr) {
  typedef typename Cx<T>::t V;
  const int n2 = c->n2, h1 = c->h1;
  if (launch_cols_ct<T>(c, inverse, planes, nplanes, zr)) {
    FVIM_CUDA_CHECK_LAUNCH();
    return FVIM_OK;
  }
  if (n2 >= 8) {
    // KC columns per CTA: 64-byte rows (full 32-byte sectors), at most 512 threads so
    // that two CTAs share an SM and overlap their loads with the other's FFT stages
    int kc = (int)(64 / sizeof(V));
    while (kc > 1 && kc * (n2 >> 3) > 512) kc >>= 1;
    if (kc > h1) kc = h1;
    const int threads = kc * (n2 >> 3);
    const size_t smem = (size_t)kc * n2 * sizeof(V);
    dim3 grid(h1 / kc, nplanes);
#define C8(INV, KCV)                                                                                  \
  if (inverse == INV && kc == KCV) {                                                                  \
    set_smem(k_cols8<T, INV, KCV>, smem);                                                             \
    k_cols8<T, INV, KCV><<<grid, threads, smem, c->stream>>>((V*)planes, (const V*)c->tw2, n2, h1);   \
  }
    C8(true, 16) C8(false, 16) C8(true, 8) C8(false, 8) C8(true, 4) C8(false, 4)
    C8(true, 2) C8(false, 2) C8(true, 1) C8(false, 1)
#undef C8
    FVIM_CUDA_CHECK_LAUNCH();
    return FVIM_OK;
  }
  // columns per CTA: 128-byte row segments when possible, within smem and item budgets
  int kc = (int)(128 / sizeof(V));
  while (kc > 1 && (size_t)kc * (n2 + 1) * sizeof(V) > 96 * 1024) kc >>= 1;
  while (kc > 1 && kc * n2 / fft_rmin(n2) > 2 * MaxT<T>::v) kc >>= 1;
  if (kc > h1) kc = h1;
  int maxi, threads;
  if (!fft_shape<T>(kc, n2, maxi, threads)) return FVIM_ERR_UNSUPPORTED;
  const size_t smem = (size_t)kc * (n2 + 1) * sizeof(V);
  dim3 grid(h1 / kc, nplanes);
#define COLS(INV, MI)                                                                              \
  if (inverse == INV && maxi == MI) {                                                              \
    set_smem(k_cols<T, INV, MI>, smem);                                                            \
    k_cols<T, INV, MI><<<grid, threads, smem, c->stream>>>((V*)planes, (const V*)c->tw2, n2, h1, kc); \
  }
  COLS(true, 2) COLS(false, 2) COLS(true, 4) COLS(false, 4)
#undef COLS
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

template <typename T> int launch_rows_inv6(const fvim_ctx* c, T* out, T nq_scale, int z0, int nzs) {
  typedef typename Cx<T>::t V;
  const int n1 = c->n1, n2 = c->n2;
  const T scale = (T)(1.0 / ((double)n1 * (double)n2));
  if (launch_rows_inv6_ct<T>(c, out, nq_scale, z0, nzs)) {
    FVIM_CUDA_CHECK_LAUNCH();
    return FVIM_OK;
  }
  if (n1 >= 8 && n1 <= 2048) {
    const int RB = r8_rows(n1, n2);
    const int threads = RB * (n1 >> 3);
    const size_t smem = (size_t)RB * 3 * (n1 + n1 / 8) * sizeof(V);
    dim3 grid(n2 / RB, nzs);
#define RI(RBV)                                                                                         \
  if (RB == RBV) {                                                                                      \
    set_smem(k_rows_inv6_r8<T, RBV>, smem);                                                             \
    k_rows_inv6_r8<T, RBV><<<grid, threads, smem, c->stream>>>((const V*)c->spec, (const T*)c->nq, out, \
                                                               (const V*)c->tw1, n1, n2, z0, nq_scale, scale); \
  }
    RI(8) RI(4) RI(2) RI(1)
#undef RI
    FVIM_CUDA_CHECK_LAUNCH();
    return FVIM_OK;
  }
  const int RB = row_block<T>(n1, n2);
  int maxi, threads;
  if (n2 % RB || !fft_shape<T>(3 * RB, n1, maxi, threads)) return FVIM_ERR_UNSUPPORTED;
  const size_t smem = (size_t)RB * 3 * n1 * sizeof(V);
  dim3 grid(n2 / RB, nzs);
  const V* spec = (const V*)c->spec;
  const T* nq = (const T*)c->nq;
  const V* tw = (const V*)c->tw1;
#define INV6(RBV, MI)                                                                                \
  if (RB == RBV && maxi == MI) {                                                                     \
    set_smem(k_rows_inv6<T, RBV, MI>, smem);                                                         \
    k_rows_inv6<T, RBV, MI><<<grid, threads, smem, c->stream>>>(spec, nq, out, tw, n1, n2, z0, nq_scale, scale); \
  }
  INV6(4, 2) INV6(2, 2) INV6(1, 2) INV6(4, 4) INV6(2, 4) INV6(1, 4)
#undef INV6
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

template <typename T> int launch_rows_inv1(const fvim_ctx* c, T* f) {
  typedef typename Cx<T>::t V;
  const int n1 = c->n1, n2 = c->n2;
  int maxi, threads;
  if (!fft_shape<T>(1, n1, maxi, threads)) return FVIM_ERR_UNSUPPORTED;
  const size_t smem = (size_t)n1 * sizeof(V);
  const T scale = (T)(1.0 / ((double)n1 * (double)n2));
  if (maxi == 2)
    k_rows_inv1<T, 2><<<n2 / 2, threads, smem, c->stream>>>((const V*)c->surf, (const T*)c->surf_nq, f,
                                                            (const V*)c->tw1, n1, n2, (T)0, scale);
  else
    k_rows_inv1<T, 4><<<n2 / 2, threads, smem, c->stream>>>((const V*)c->surf, (const T*)c->surf_nq, f,
                                                            (const V*)c->tw1, n1, n2, (T)0, scale);
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

template int launch_rows_fwd6<float>(const fvim_ctx*, const float*, int, int, const int*);
template int launch_rows_fwd6<double>(const fvim_ctx*, const double*, int, int, const int*);
template int launch_rows_fwd1<float>(const fvim_ctx*, const float*);
template int launch_rows_fwd1<double>(const fvim_ctx*, const double*);
template int launch_cols<float>(const fvim_ctx*, bool, void*, int, const int*);
template int launch_cols<double>(const fvim_ctx*, bool, void*, int, const int*);
template int launch_rows_inv6<float>(const fvim_ctx*, float*, float, int, int);
template int launch_rows_inv6<double>(const fvim_ctx*, double*, double, int, int);
template int launch_rows_inv1<float>(const fvim_ctx*, float*);
template int launch_rows_inv1<double>(const fvim_ctx*, double*);

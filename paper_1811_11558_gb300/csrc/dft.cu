// In-plane discrete Fourier transforms of grids whose sides are not both powers of two (odd
// sides such as 81 = 3^4, the discretisation of the paper's elastic-perfectly-plastic Hertz
// comparison, App. C).  Direct evaluation of the Sec. 3.1 DFT,
//   X(k) = sum_n x(n) exp(-2 pi i k n / N),
// O(N) per output value, with the exact twiddle table exp(-2 pi i j / N), j = (k n) mod N.
//
// Layout (fvim_ctx::gen): the half spectrum of a real row keeps k1 = 0 .. floor(N1/2) (hs
// columns; for an even N1 the last one is the Nyquist column, which the depth kernel treats
// as outside Z^2_N), stored with a row stride ldh = hs rounded up to 16 columns; the padding
// columns are written as zeros.  There is no side array: every coefficient is in the
// spectrum.  The full spectrum of a real row follows from X(N1 - k) = conj X(k).
//
// These kernels serve grids up to a few hundred points per side, where O(N^2) per line is a
// small cost next to the depth operator; power-of-two grids take the FFT kernels.
#include "fvim_internal.cuh"

namespace {

constexpr int RB = 4;     // rows per CTA (row kernels)
constexpr int CT = 16;    // columns per CTA (column kernel)

// forward row DFTs of real rows: src [rows][n1] -> dst [rows][ldh] (k1 < hs, zeros above)
template <typename T>
__global__ void __launch_bounds__(128) k_dft_rows_fwd(const T* __restrict__ src, typename Cx<T>::t* __restrict__ dst,
                                                      const typename Cx<T>::t* __restrict__ tw, int n1, int hs,
                                                      int ldh, size_t rows) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* w = reinterpret_cast<V*>(smraw);                 // [n1] twiddles
  T* x = reinterpret_cast<T*>(w + n1);                // [RB][n1]
  const size_t r0 = (size_t)blockIdx.x * RB;
  const int nr = (int)((rows - r0) < (size_t)RB ? rows - r0 : RB);
  for (int i = threadIdx.x; i < n1; i += blockDim.x) w[i] = tw[i];
  for (int i = threadIdx.x; i < nr * n1; i += blockDim.x) x[i] = src[r0 * n1 + i];
  __syncthreads();
  for (int i = threadIdx.x; i < nr * ldh; i += blockDim.x) {
    const int r = i / ldh, k = i - r * ldh;
    V acc = mk<V>(0, 0);
    if (k < hs) {
      const T* xr = x + r * n1;
      int j = 0;  // (k n) mod n1
      for (int n = 0; n < n1; ++n) {
        acc = caxpy(acc, xr[n], w[j]);
        j += k;
        if (j >= n1) j -= n1;
      }
    }
    dst[(r0 + r) * ldh + k] = acc;
  }
}

// column DFTs along x2, in place: planes [nplanes][n2][ldh], CT columns per CTA (the tile and
// its transform both in shared memory)
template <typename T, bool INV>
__global__ void __launch_bounds__(256) k_dft_cols(typename Cx<T>::t* __restrict__ spec,
                                                  const typename Cx<T>::t* __restrict__ tw, int n2, int ldh) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* w = reinterpret_cast<V*>(smraw);       // [n2] twiddles
  V* a = w + n2;                            // [n2][CT] the CTA's columns
  V* b = a + (size_t)n2 * CT;               // [n2][CT] their transforms
  V* P = spec + (size_t)blockIdx.y * n2 * ldh + (size_t)blockIdx.x * CT;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    V t = tw[i];
    if (INV) t.y = -t.y;
    w[i] = t;
  }
  for (int i = threadIdx.x; i < n2 * CT; i += blockDim.x) {
    const int row = i / CT, c = i - row * CT;
    a[i] = P[(size_t)row * ldh + c];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n2 * CT; i += blockDim.x) {
    const int k = i / CT, c = i - k * CT;
    int j = 0;  // (k n) mod n2
    V acc = mk<V>(0, 0);
    for (int n = 0; n < n2; ++n) {
      acc = cadd(acc, cmul(a[n * CT + c], w[j]));
      j += k;
      if (j >= n2) j -= n2;
    }
    b[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n2 * CT; i += blockDim.x) {
    const int row = i / CT, c = i - row * CT;
    P[(size_t)row * ldh + c] = b[i];
  }
}

// inverse row DFTs to real rows: src [rows][ldh] (k1 < hs) -> dst [rows][n1], times scale;
// x(n) = X(0) + 2 sum_{0 < k < n1/2} Re(X(k) e^{2 pi i k n / n1}) + (n1 even) X(n1/2) (-1)^n
template <typename T>
__global__ void __launch_bounds__(128) k_dft_rows_inv(const typename Cx<T>::t* __restrict__ src, T* __restrict__ dst,
                                                      const typename Cx<T>::t* __restrict__ tw, int n1, int hs,
                                                      int ldh, size_t rows, T scale) {
  typedef typename Cx<T>::t V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* w = reinterpret_cast<V*>(smraw);   // [n1]
  V* X = w + n1;                        // [RB][hs]
  const size_t r0 = (size_t)blockIdx.x * RB;
  const int nr = (int)((rows - r0) < (size_t)RB ? rows - r0 : RB);
  for (int i = threadIdx.x; i < n1; i += blockDim.x) w[i] = tw[i];
  for (int i = threadIdx.x; i < nr * hs; i += blockDim.x) {
    const int r = i / hs, k = i - r * hs;
    X[i] = src[(r0 + r) * ldh + k];
  }
  __syncthreads();
  const bool even = (n1 & 1) == 0;
  const int kmax = even ? n1 / 2 - 1 : (n1 - 1) / 2;  // last k with a conjugate partner
  for (int i = threadIdx.x; i < nr * n1; i += blockDim.x) {
    const int r = i / n1, n = i - r * n1;
    const V* Xr = X + r * hs;
    T acc = Xr[0].x;
    int j = n;  // (k n) mod n1 for k = 1
    T s = 0;
    for (int k = 1; k <= kmax; ++k) {
      // Re(X e^{+i theta}) with tw = e^{-i theta}: X.x tw.x + X.y tw.y
      s += Xr[k].x * w[j].x + Xr[k].y * w[j].y;
      j += n;
      if (j >= n1) j -= n1;
    }
    acc += 2 * s;
    if (even) acc += (n & 1) ? -Xr[n1 / 2].x : Xr[n1 / 2].x;
    dst[(r0 + r) * n1 + n] = acc * scale;
  }
}

}  // namespace

template <typename T> int launch_dft_rows_fwd(const fvim_ctx* c, const T* src, void* dst, size_t rows) {
  typedef typename Cx<T>::t V;
  const size_t smem = (size_t)c->n1 * sizeof(V) + (size_t)RB * c->n1 * sizeof(T);
  smem_cap(k_dft_rows_fwd<T>);
  k_dft_rows_fwd<T><<<(unsigned)((rows + RB - 1) / RB), 128, smem, c->stream>>>(src, (V*)dst, (const V*)c->tw1, c->n1,
                                                                                c->hs, c->h1, rows);
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

template <typename T> int launch_dft_cols(const fvim_ctx* c, bool inverse, void* planes, int nplanes) {
  typedef typename Cx<T>::t V;
  const size_t smem = (size_t)c->n2 * sizeof(V) + (size_t)2 * c->n2 * CT * sizeof(V);
  dim3 grid(c->h1 / CT, nplanes);
  if (inverse) {
    smem_cap(k_dft_cols<T, true>);
    k_dft_cols<T, true><<<grid, 256, smem, c->stream>>>((V*)planes, (const V*)c->tw2, c->n2, c->h1);
  } else {
    smem_cap(k_dft_cols<T, false>);
    k_dft_cols<T, false><<<grid, 256, smem, c->stream>>>((V*)planes, (const V*)c->tw2, c->n2, c->h1);
  }
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

template <typename T> int launch_dft_rows_inv(const fvim_ctx* c, const void* src, T* dst, size_t rows, T scale) {
  typedef typename Cx<T>::t V;
  const size_t smem = (size_t)c->n1 * sizeof(V) + (size_t)RB * c->hs * sizeof(V);
  smem_cap(k_dft_rows_inv<T>);
  k_dft_rows_inv<T><<<(unsigned)((rows + RB - 1) / RB), 128, smem, c->stream>>>((const V*)src, dst, (const V*)c->tw1,
                                                                                c->n1, c->hs, c->h1, rows, scale);
  FVIM_CUDA_CHECK_LAUNCH();
  return FVIM_OK;
}

template int launch_dft_rows_fwd<float>(const fvim_ctx*, const float*, void*, size_t);
template int launch_dft_rows_fwd<double>(const fvim_ctx*, const double*, void*, size_t);
template int launch_dft_cols<float>(const fvim_ctx*, bool, void*, int);
template int launch_dft_cols<double>(const fvim_ctx*, bool, void*, int);
template int launch_dft_rows_inv<float>(const fvim_ctx*, const void*, float*, size_t, float);
template int launch_dft_rows_inv<double>(const fvim_ctx*, const void*, double*, size_t, double);

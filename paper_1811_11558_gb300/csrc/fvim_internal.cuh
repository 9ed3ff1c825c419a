// Internal definitions shared by the CUDA translation units of libfvim.
// Not part of the public ABI (see include/fvim.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fvim.h"

// ---------------------------------------------------------------------------
// complex helpers (float2 / double2)
// ---------------------------------------------------------------------------
template <typename T> struct Cx;
template <> struct Cx<float> { typedef float2 t; };
template <> struct Cx<double> { typedef double2 t; };

template <typename V> __host__ __device__ __forceinline__ V mk(decltype(V::x) a, decltype(V::x) b) {
  V r; r.x = a; r.y = b; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return mk<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return mk<V>(a.x * s, a.y * s); }
// multiply by i
template <typename V> __device__ __forceinline__ V cmuli(V a) { return mk<V>(-a.y, a.x); }
// a + s*b (s real)
template <typename V> __device__ __forceinline__ V caxpy(V a, decltype(V::x) s, V b) {
  return mk<V>(a.x + s * b.x, a.y + s * b.y);
}
// a + s*i*b (s real): two scalar multiply-adds, the swap and the sign folded into them
template <typename V> __device__ __forceinline__ V caxpy_i(V a, decltype(V::x) s, V b) {
  return mk<V>(a.x - s * b.y, a.y + s * b.x);
}

#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000) && !defined(FVIM_NO_F32X2)
// Blackwell packed FP32 pairs (add/sub/mul/fma .f32x2): one instruction per FP32 complex
// add, subtract, real scale or real axpy, each lane rounded as its scalar counterpart.
__device__ __forceinline__ unsigned long long f2pack(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 f2unpack(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pack(a)), "l"(f2pack(b)));
  return f2unpack(d);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pack(a)), "l"(f2pack(b)));
  return f2unpack(d);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pack(a)), "l"(f2pack(make_float2(s, s))));
  return f2unpack(d);
}
__device__ __forceinline__ float2 caxpy(float2 a, float s, float2 b) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2pack(make_float2(s, s))), "l"(f2pack(b)), "l"(f2pack(a)));
  return f2unpack(d);
}
#endif

// ---------------------------------------------------------------------------
// Shared-memory FFT: batched, in place, Stockham autosort with radix 8/4/2
// stages.  Every thread of the block takes part; at most MAXI work items (one
// radix-R butterfly each) per thread and stage, so the caller must launch at
// least ceil(nfft * n / rmin(n) / MAXI) threads.  tw[k] = exp(-2 pi i k / n).
// ---------------------------------------------------------------------------
__host__ __device__ inline int fft_radix(int m) {
  // radix of the next stage for a remaining length m (plans 8..8 then 4/4 or 4 or 2)
  if (m == 2) return 2;
  if (m == 4) return 4;
  if (m == 16) return 4;           // 16 = 4 x 4 instead of 8 x 2
  if (m % 8 == 0) return 8;
  return 4;
}
__host__ __device__ inline int fft_rmin(int n) {
  int rmin = 8, m = n;
  while (m > 1) { int r = fft_radix(m); if (r < rmin) rmin = r; m /= r; }
  return rmin;
}

template <typename V, bool INV>
__device__ __forceinline__ V twiddle(const V* tw, int idx) {
  V w = tw[idx];
  if (INV) w.y = -w.y;
  return w;
}

template <typename V, bool INV>
__device__ __forceinline__ void dft2(V& a, V& b) { V t = a; a = cadd(t, b); b = csub(t, b); }

template <typename V, bool INV>
__device__ __forceinline__ void dft4(V* v) {
  V a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
  V b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
  v[0] = cadd(a0, b0);
  v[2] = csub(a0, b0);
  // a1 -/+ i b1 (forward W4 = -i, inverse +i), the swap folded into the adds
  if (INV) {
    v[1] = mk<V>(a1.x - b1.y, a1.y + b1.x);
    v[3] = mk<V>(a1.x + b1.y, a1.y - b1.x);
  } else {
    v[1] = mk<V>(a1.x + b1.y, a1.y - b1.x);
    v[3] = mk<V>(a1.x - b1.y, a1.y + b1.x);
  }
}

template <typename V, bool INV>
__device__ __forceinline__ void dft8(V* v) {
  typedef decltype(V::x) T;
  const T r = (T)0.70710678118654752440;
  V e[4] = {v[0], v[2], v[4], v[6]};
  V o[4] = {v[1], v[3], v[5], v[7]};
  dft4<V, INV>(e);
  dft4<V, INV>(o);
  // twiddles W8^m, m = 0..3 (forward exp(-i pi m/4)): products by r(1 -/+ i), -/+ i and
  // r(-1 -/+ i) written out (the zero parts of the twiddles cost nothing)
  const V o1 = o[1], o2 = o[2], o3 = o[3];
  if (INV) {
    o[1] = mk<V>(r * (o1.x - o1.y), r * (o1.x + o1.y));
    o[2] = mk<V>(-o2.y, o2.x);
    o[3] = mk<V>(-r * (o3.x + o3.y), r * (o3.x - o3.y));
  } else {
    o[1] = mk<V>(r * (o1.x + o1.y), r * (o1.y - o1.x));
    o[2] = mk<V>(o2.y, -o2.x);
    o[3] = mk<V>(r * (o3.y - o3.x), -r * (o3.x + o3.y));
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    v[m] = cadd(e[m], o[m]);
    v[m + 4] = csub(e[m], o[m]);
  }
}

template <typename V, bool INV, int R, int MAXI>
__device__ __forceinline__ void fft_stage(V* buf, int n, int nfft, int fstride, int Ns, const V* tw) {
  const int per = n / R;
  const int items = nfft * per;
  V v[MAXI][R];
#pragma unroll
  for (int it = 0; it < MAXI; ++it) {
    const int w = threadIdx.x + it * blockDim.x;
    if (w < items) {
      const int f = w / per, j = w - f * per;
      const V* b = buf + (size_t)f * fstride;
#pragma unroll
      for (int r = 0; r < R; ++r) v[it][r] = b[j + r * per];
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < MAXI; ++it) {
    const int w = threadIdx.x + it * blockDim.x;
    if (w < items) {
      const int f = w / per, j = w - f * per;
      const int k = j % Ns;
      const int step = n / (Ns * R);
#pragma unroll
      for (int r = 1; r < R; ++r) v[it][r] = cmul(v[it][r], twiddle<V, INV>(tw, (r * k * step) & (n - 1)));
      if (R == 8) dft8<V, INV>(v[it]);
      else if (R == 4) dft4<V, INV>(v[it]);
      else dft2<V, INV>(v[it][0], v[it][1]);
      V* b = buf + (size_t)f * fstride;
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) b[base + r * Ns] = v[it][r];
    }
  }
  __syncthreads();
}

// nfft transforms of length n (power of two >= 2) in shared memory, FFT f at
// buf + f * fstride.  Unnormalised; INV uses exp(+2 pi i k/n).
template <typename V, bool INV, int MAXI>
__device__ void block_fft(V* buf, int n, int nfft, int fstride, const V* tw) {
  int Ns = 1;
  int m = n;
  while (m > 1) {
    const int R = fft_radix(m);
    if (R == 8) fft_stage<V, INV, 8, MAXI>(buf, n, nfft, fstride, Ns, tw);
    else if (R == 4) fft_stage<V, INV, 4, MAXI>(buf, n, nfft, fstride, Ns, tw);
    else fft_stage<V, INV, 2, MAXI>(buf, n, nfft, fstride, Ns, tw);
    Ns *= R;
    m /= R;
  }
}

// ---------------------------------------------------------------------------
// Register-resident Stockham FFT (n >= 8): thread t of an FFT holds the 8 strided
// elements x[t + m n/8], m = 0..7, for the whole transform.  A stage of radix R
// (8, 4 or 2; plan of fft_radix) runs 1, 2 or 4 butterflies per thread on those
// registers and reports, for every register slot, the natural index its result
// belongs to; between stages the values go through shared memory.  After the last
// stage slot m holds the output at index t + m n/8 (natural order).
// ---------------------------------------------------------------------------
template <typename V, bool INV>
__device__ __forceinline__ void reg_stage(V (&v)[8], int (&pos)[8], int t, int n, int R, int Ns, const V* tw) {
  const int T8 = n >> 3;
  if (R == 8) {
    const int k = t & (Ns - 1);
    const int step = n / (Ns * 8);
#pragma unroll
    for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], twiddle<V, INV>(tw, (r * k * step) & (n - 1)));
    dft8<V, INV>(v);
    const int base = (t / Ns) * Ns * 8 + k;
#pragma unroll
    for (int r = 0; r < 8; ++r) pos[r] = base + r * Ns;
  } else if (R == 4) {
    const int step = n / (Ns * 4);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int b = t + g * T8;
      const int k = b & (Ns - 1);
      V u[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) u[r] = v[2 * r + g];
#pragma unroll
      for (int r = 1; r < 4; ++r) u[r] = cmul(u[r], twiddle<V, INV>(tw, (r * k * step) & (n - 1)));
      dft4<V, INV>(u);
      const int base = (b / Ns) * Ns * 4 + k;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        v[2 * r + g] = u[r];
        pos[2 * r + g] = base + r * Ns;
      }
    }
  } else {
    const int step = n / (Ns * 2);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int b = t + m * T8;
      const int k = b & (Ns - 1);
      V a = v[m], c = cmul(v[m + 4], twiddle<V, INV>(tw, (k * step) & (n - 1)));
      v[m] = cadd(a, c);
      v[m + 4] = csub(a, c);
      const int base = (b / Ns) * Ns * 2 + k;
      pos[m] = base;
      pos[m + 4] = base + Ns;
    }
  }
}

// ---------------------------------------------------------------------------
// The same register-resident Stockham FFT with the length N known at compile time:
// the stage list is unrolled, the first stage has no twiddles, and every index is a
// shift or a mask.  NF transforms per thread share each shared-memory exchange; the
// exchange layout is the caller's (Sm::put / Sm::get).  After the call slot m of
// transform f holds the output at index t + m N/8.
// ---------------------------------------------------------------------------
template <int REM> struct StageRadix {
  static constexpr int v = (REM == 2) ? 2 : ((REM == 4 || REM == 16) ? 4 : ((REM % 8 == 0) ? 8 : 4));
};

// twiddles w^1..w^7 of a radix-8 butterfly (w = tw[idx]) from three table reads: w, w^2, w^4
// are read, w^3 = w w^2, w^5 = w^4 w, w^6 = w^4 w^2, w^7 = w^4 w^3 (three table reads instead of
// seven: the reads of one stage are scattered, a table read per product was the costly part)
template <typename V, bool INV>
__device__ __forceinline__ void twiddles8(const V* __restrict__ tw, int idx, V (&w)[8]) {
  w[1] = twiddle<V, INV>(tw, idx);
  w[2] = twiddle<V, INV>(tw, 2 * idx);
  w[4] = twiddle<V, INV>(tw, 4 * idx);
  w[3] = cmul(w[1], w[2]);
  w[5] = cmul(w[4], w[1]);
  w[6] = cmul(w[4], w[2]);
  w[7] = cmul(w[4], w[3]);
}

template <typename V, bool INV, int N, int R, int NS>
__device__ __forceinline__ void stage_ct(V (&v)[8], int (&pos)[8], int t, const V* __restrict__ tw) {
  constexpr int T8 = N / 8;
  if constexpr (R == 8) {
    const int k = t & (NS - 1);
    if constexpr (NS > 1) {
      constexpr int step = N / (NS * 8);
      V w[8];
      twiddles8<V, INV>(tw, k * step, w);
#pragma unroll
      for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], w[r]);
    }
    dft8<V, INV>(v);
    const int base = (t / NS) * NS * 8 + k;
#pragma unroll
    for (int r = 0; r < 8; ++r) pos[r] = base + r * NS;
  } else if constexpr (R == 4) {
    constexpr int step = N / (NS * 4);
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int b = t + g * T8;
      const int k = b & (NS - 1);
      V u[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) u[r] = v[2 * r + g];
      if constexpr (NS > 1) {
        // w, w^2 read, w^3 = w w^2
        const V w1 = twiddle<V, INV>(tw, k * step), w2 = twiddle<V, INV>(tw, 2 * k * step);
        u[1] = cmul(u[1], w1);
        u[2] = cmul(u[2], w2);
        u[3] = cmul(u[3], cmul(w1, w2));
      }
      dft4<V, INV>(u);
      const int base = (b / NS) * NS * 4 + k;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        v[2 * r + g] = u[r];
        pos[2 * r + g] = base + r * NS;
      }
    }
  } else {
    constexpr int step = N / (NS * 2);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int b = t + m * T8;
      const int k = b & (NS - 1);
      V c = v[m + 4];
      if constexpr (NS > 1) c = cmul(c, twiddle<V, INV>(tw, k * step));
      const V a = v[m];
      v[m] = cadd(a, c);
      v[m + 4] = csub(a, c);
      const int base = (b / NS) * NS * 2 + k;
      pos[m] = base;
      pos[m + 4] = base + NS;
    }
  }
}

// barrier over the whole CTA (the default exchange synchronisation of fft_ct)
struct CtaSync {
  __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
// barrier over a group of NG threads (a multiple of 32, whole warps): the warp itself, or a
// named barrier id (1..15) shared by the group's warps only
template <int NG> struct GroupSync {
  int id;
  __device__ __forceinline__ void operator()() const {
    if constexpr (NG == 32) {
      __syncwarp();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(NG) : "memory");
    }
  }
};

template <typename V, bool INV, int N, int NF, int NS, class Sm, class Sync = CtaSync>
__device__ __forceinline__ void fft_ct(V (&v)[NF][8], int t, const Sm& sm, const V* __restrict__ tw,
                                       const Sync& sync = Sync()) {
  constexpr int R = StageRadix<N / NS>::v;
  int pos[8];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    stage_ct<V, INV, N, R, NS>(v[f], pos, t, tw);
    if constexpr (NS * R < N) {
#pragma unroll
      for (int m = 0; m < 8; ++m) sm.put(f, pos[m], v[f][m]);
    }
  }
  if constexpr (NS * R < N) {
    sync();
#pragma unroll
    for (int f = 0; f < NF; ++f)
#pragma unroll
      for (int m = 0; m < 8; ++m) v[f][m] = sm.get(f, t + m * (N / 8));
    sync();
    fft_ct<V, INV, N, NF, NS * R>(v, t, sm, tw, sync);
  }
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async), all in flight before one wait
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
template <typename V> __device__ __forceinline__ void cp_async_cx(V* smem, const V* gmem) {
  if (sizeof(V) == 16) cp_async_16(smem, gmem);
  else cp_async_8(smem, gmem);
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// wait until at most N of this thread's committed copy groups are still in flight
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Raises a kernel's dynamic shared-memory cap to the device's opt-in maximum.  The value is
// the same on every call: contexts used from several host threads launch one kernel with
// different sizes, and a cap set to the exact size of one launch could be lowered under
// another thread's launch of the same kernel.
inline int smem_optin_max() {
  static const int v = [] {
    int dev = 0, m = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return m > 0 ? m : 48 * 1024;
  }();
  return v;
}
template <typename K> inline void smem_cap(K kern) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_max());
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
#define FVIM_NSOLVER_BUFS 26

struct fvim_ctx {
  // h1: row stride of the half spectrum (complex); power-of-two grids: N1/2 columns (the
  // k1 = N1/2 coefficient kept apart in nq); gen: floor(N1/2) + 1 columns rounded up to 16
  int n1, n2, nz, h1;
  int gen;  // a side is not a power of two: direct DFTs (dft.cu), every coefficient in spec
  int hs;   // stored k1 columns (k1 < hs); == h1 for power-of-two grids
  int prec;  // FVIM_FP32 / FVIM_FP64
  double L1, L2;
  double E, nu, sigma_y, E_h, lam, mu;
  cudaStream_t stream;
  int device;
  int uniform;   // depth nodes equally spaced
  double hz;     // spacing when uniform
  double* z_host;
  void* z_dev;   // T[nz]
  void* tw1;     // complex T[n1]
  void* tw2;     // complex T[n2]
  void* spec;    // complex T[nz][6][n2][h1]
  void* nq;      // T[nz][6][n2] row-Nyquist coefficients
  void* surf;    // complex T[n2][h1]
  void* surf_nq; // T[n2]
  void* st_eps_p; // T[nz][6][n2][n1]
  void* st_ep;    // T[nz][n2][n1]
  void* st_sig;   // T[nz][6][n2][n1]
  void* st_T;     // T[n2][n1] contact pressure of the last converged increment
  int last_kernels;
  void* prof;  // ProfState* (capi.cu) or NULL
  // solver workspace (solvers.cu), allocated on first use
  void* sv[FVIM_NSOLVER_BUFS];
  double* h_part;  // host copy of reduction partials
  long n_applies;  // Mindlin applies issued by the solvers
  int fft2_cl;     // whole-plane cluster FFTs usable: -1 not yet known, 0 no, 1 yes
  void* srt;       // solver runtime (solvers.cu): own stream, events, captured CUDA graphs
  int depth_chunk; // depth nodes per chunk thread of the depth kernel; 0: depth_chunk_default
  int plan_tuned;  // depth_chunk came from a timing run (fvim_autotune) in this process
  int depth_ctas;  // CTAs per SM of the FP32 register depth kernel: 0 or 2 (128 registers), 3 (85)
  float depth_cut; // chunk-scan cutoff eps_co of the FP32 register depth kernel (0: exact scan)
  void* tmap;      // CUtensorMap (host, 64-byte aligned) over the spectrum for the depth tile, or NULL
  int tma_rows;    // rows (z, component) per tensor-copy box of the depth tile; 0: no tensor copies
  int* dev_status; // device status word: bit 0 set by a bounded device wait that expired
  int tma_test_extra;  // bytes added to the depth tile's expected copy count (tests of the
                       // expired-wait path only; FVIM_TEST_TMA_EXTRA at creation, else 0)
  int fft2_fused;  // one-pass 2-D FFTs through L2: -1 not yet known, 0 not used, 1 used
  int fft_path;    // in-plane FFT path chosen by the tuner or fvim_set_plan (FVIM_FFT_*), -1: none
                   // (the row / column kernels unless an environment variable selects another)
};

// tile plan of the depth kernel (depth.cu): default chunk length, and whether a chunk length
// gives a launchable configuration on this context's grid and precision
int depth_chunk_default(int nz);
// ctas: CTAs per SM the FP32 register variant is compiled for (2 default, 3 with 85 registers)
bool depth_chunk_ok(const fvim_ctx* c, int chunk, int ctas = 2);
// CTAs per SM of the depth kernel's launch under the context's plan (0: shared-memory variant)
int depth_launch_ctas(const fvim_ctx* c);
// process-wide plan table (tune.cu): the tuned chunk length of a grid, or 0; its tuned FFT
// path, or -1
int plan_lookup(const fvim_ctx* c);
int plan_lookup_fft(const fvim_ctx* c);
int plan_lookup_ctas(const fvim_ctx* c);
// whether an in-plane FFT path is built for the context's grid and precision (capi.cu)
bool fft_path_available(const fvim_ctx* c, int path);

// kernel kinds for fvim_profile_read
enum ProfSlot {
  PROF_ROWS_FWD6 = 0, PROF_COLS_FWD, PROF_MINDLIN_DEPTH, PROF_COLS_INV, PROF_ROWS_INV6,
  PROF_ROWS_FWD1, PROF_ROWS_INV1, PROF_BOUSSINESQ, PROF_RETURN_MAP, PROF_COMMIT, PROF_FFT2_FWD,
  PROF_FFT2_INV, PROF_NSLOTS
};

// material constants handed to kernels
template <typename T> struct Mat {
  T lam, mu, nu, sigma_y, E_h;
};

// launchers (defined in the .cu files, instantiated for float and double)
// zr (device, two ints) or NULL: only layers zr[0] <= z < zr[1] hold non-zero input; the forward
// passes skip the others and the depth kernel reads them as zero
template <typename T> int launch_rows_fwd6(const fvim_ctx* c, const T* eps_p, int z0, int nzs, const int* zr = nullptr);
template <typename T> int launch_rows_fwd1(const fvim_ctx* c, const T* f);
template <typename T> int launch_cols(const fvim_ctx* c, bool inverse, void* planes, int nplanes, const int* zr = nullptr);
template <typename T> int launch_rows_inv6(const fvim_ctx* c, T* out, T nq_scale, int z0, int nzs);
template <typename T> int launch_rows_inv1(const fvim_ctx* c, T* f);
// eps_in: the spectrum holds eps_p (Hooke's law applied per mode) instead of w = C:eps_p
template <typename T>
int launch_mindlin_depth(const fvim_ctx* c, int out_kind, bool want_u3, bool eps_in = false, const int* zr = nullptr);
template <typename T> int launch_boussinesq(const fvim_ctx* c, int out_kind, bool want_vol, bool want_u3);
template <typename T> int launch_return_map(const fvim_ctx* c, const T* d_eps, T* d_eps_p, T* d_ep);
template <typename T> int launch_commit(const fvim_ctx* c, const T* d_eps, const T* d_eps_p, const T* d_ep);
template <typename T> int launch_zero_nq(const fvim_ctx* c);

// solver runtime (solvers.cu): release, and drop captured graphs after a material change
void solver_release(fvim_ctx* c);
void solver_drop_graphs(fvim_ctx* c);

// whole-plane cluster FFTs (fft2d_cluster.cu), FP32 and a few plane sizes only
bool fft2_cluster_available(const fvim_ctx* c);
int launch_fft2_fwd_cluster(const fvim_ctx* c, const float* src);
int launch_fft2_inv_cluster(const fvim_ctx* c, float* out, int nq_mode, float nq_scale);

// one-pass 2-D FFTs with the row spectra exchanged through L2 (fft2d_l2.cu), FP32; zr as for
// launch_rows_fwd6 (planes of layers outside the range are skipped)
bool fft2_fused_available(const fvim_ctx* c);
int launch_fft2_fwd_fused(const fvim_ctx* c, const float* src, const int* zr = nullptr);
int launch_fft2_inv_fused(const fvim_ctx* c, float* out, int nq_mode, float nq_scale);

// direct DFTs of grids with a side that is not a power of two (dft.cu, fvim_ctx::gen):
// rows real -> half spectrum [rows][h1], columns in place, half spectrum -> real rows x scale
template <typename T> int launch_dft_rows_fwd(const fvim_ctx* c, const T* src, void* dst, size_t rows);
template <typename T> int launch_dft_cols(const fvim_ctx* c, bool inverse, void* planes, int nplanes);
template <typename T> int launch_dft_rows_inv(const fvim_ctx* c, const void* src, T* dst, size_t rows, T scale);
// grid sides the library takes: a power of two (4..1024 for N1, 2..1024 for N2, the FFT path)
// or an odd number 3..255 (with the other side odd or a power of two up to 256: direct DFTs)
bool grid_ok(int n1, int n2);
bool grid_gen(int n1, int n2);
int spec_stride(int n1, int n2);

// compile-time-length FFT kernels (fft_ct.cu); false when the length has no variant
template <typename T> bool launch_cols_ct(const fvim_ctx* c, bool inverse, void* planes, int nplanes, const int* zr = nullptr);
// surface compliance applied in the column pass (fft_ct.cu); false when N2 has no variant
template <typename T> bool launch_cols_conv_ct(const fvim_ctx* c);
template <typename T> bool launch_rows_fwd6_ct(const fvim_ctx* c, const T* eps_p, int z0, int nzs, const int* zr = nullptr);
template <typename T> bool launch_rows_inv6_ct(const fvim_ctx* c, T* out, T nq_scale, int z0, int nzs);

// ---- J2 radial return with linear isotropic hardening (Sec. 4.1) at one voxel -----------
// de: strain increment, sig: stress of the last converged increment, ep: cumulated plastic
// strain there.  Returns the increment of cumulated plastic strain and writes the plastic
// strain increment (Voigt order 11, 22, 33, 23, 13, 12; shear entries are tensor components).
// Shared by the return-map kernel and the fused DF-SANE trial kernel (the same arithmetic).
template <typename T>
__device__ __forceinline__ T rmap_voxel(const T (&de)[6], const T (&sig)[6], T ep, T lam, T mu, T sy, T Eh,
                                        T (&dp)[6]) {
  T st[6];
  const T tr = de[0] + de[1] + de[2];
#pragma unroll
  for (int c = 0; c < 6; ++c) st[c] = sig[c] + 2 * mu * de[c];
  st[0] += lam * tr;
  st[1] += lam * tr;
  st[2] += lam * tr;
  const T m = (st[0] + st[1] + st[2]) / (T)3;
  const T s[6] = {st[0] - m, st[1] - m, st[2] - m, st[3], st[4], st[5]};
  const T nrm2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + 2 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
  const T fy = sqrt((T)1.5 * nrm2);
  const T f = fy - (sy + Eh * ep);
  T dEp = 0, k = 0;
  if (f > 0) {
    dEp = f / ((T)3 * mu + Eh);
    k = (T)1.5 * dEp / fy;
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) dp[c] = k * s[c];
  return dEp;
}

// layer range of the flowing voxels (elsewhere the plastic increment is exactly zero): one
// pair of atomics per warp, over the lanes that flow
__device__ __forceinline__ void flow_range_note(int* zr, int z) {
  const unsigned am = __activemask();
  const int lo = __reduce_min_sync(am, z), hi = __reduce_max_sync(am, z);
  if ((int)(threadIdx.x & 31) == __ffs(am) - 1) {
    atomicMin(zr, lo);
    atomicMax(zr + 1, hi + 1);
  }
}

// ---- grouped Mindlin apply: FP32 problems of uneven size, one launch per phase ----------
// One problem of a group: its context's buffers and the constants its kernels need.
constexpr int kGrpMax = 64;  // problems per group (the table travels as a kernel parameter)
struct GrpProb {
  const float* eps;      // eps_p [nz][6][n2][n1]
  float* out;            // stress or strain [nz][6][n2][n1]
  float2* spec;          // half spectrum [nz][6][n2][h1]
  float* nq;             // k1 = N1/2 coefficients [nz][6][n2]
  const float2* tw1;     // twiddles of N1
  const float2* tw2;     // twiddles of N2
  const float* zn;       // depth nodes [nz]
  int n1, n2, nz, h1, hs;
  int nch, nchp;         // depth chunks of 4 nodes, and that count rounded up to a power of two
  int uniform, out_kind;
  float w1, w2, lam, mu, nu, hz, cut;
  float nq_scale, scale; // inverse rows: Nyquist factor and 1 / (N1 N2)
};
struct GrpTable {
  int n;                     // problems
  int start[kGrpMax + 1];    // first CTA of each problem in the launch; start[n] = CTAs
  GrpProb p[kGrpMax];
};
static_assert(sizeof(GrpTable) < 16 * 1024, "the group table is a kernel parameter");
// the problem of CTA b: the last i with start[i] <= b
__device__ __forceinline__ int grp_find(const GrpTable& t, int b) {
  int lo = 0, hi = t.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
// the four kinds of grouped launch (fft_ct.cu, depth.cu); each fills t.start for its own CTA
// counts.  Problems: FP32, 64 <= N1, N2 <= 512 powers of two, Nz <= 64.
int launch_grp_rows_fwd(GrpTable& t, cudaStream_t s);
int launch_grp_cols(GrpTable& t, bool inverse, cudaStream_t s);
int launch_grp_depth(GrpTable& t, cudaStream_t s);
int launch_grp_rows_inv(GrpTable& t, cudaStream_t s);

// launch sequences of the entry points (capi.cu), used by the solvers
// zr: see launch_rows_fwd6; honoured for FVIM_STRAIN output only
template <typename T> int apply_mindlin_t(fvim_ctx* c, const T* eps_p, T* out, int kind, T* u3, const int* zr = nullptr);
template <typename T> int apply_boussinesq_t(fvim_ctx* c, const T* p, T* u3, T* vol, int kind);
// zr (device, two ints) or NULL: receives the layer range [zr[0], zr[1]) of the voxels that
// flow (reset by the caller to {INT_MAX-ish, 0} first).
template <typename T> int return_map_t(fvim_ctx* c, const T* d_eps, T* d_eps_p, T* d_ep, int* zr = nullptr);
template <typename T> int commit_t(fvim_ctx* c, const T* d_eps, const T* d_eps_p, const T* d_ep);

// true when e is an error; the error and the source line that saw it are kept as this host
// thread's last CUDA error (fvim_last_cuda_error)
bool fvim_cuda_failed(cudaError_t e, const char* file = nullptr, int line = 0);
#define FVIM_CU(call) fvim_cuda_failed((call), __FILE__, __LINE__)
#define FVIM_CUDA_CHECK_LAUNCH()                                                        \
  do {                                                                                  \
    if (fvim_cuda_failed(cudaGetLastError(), __FILE__, __LINE__)) return FVIM_ERR_CUDA; \
  } while (0)

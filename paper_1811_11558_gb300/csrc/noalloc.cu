// Allocation-free variant of the Mindlin-operator apply (see fvim_apply_mindlin_noalloc
// in include/fvim.h).
//
// Some callers cannot allocate device memory once they are running: a host framework
// that owns every device allocation through its own pool, a latency-critical service
// that must not hit cudaMalloc/cudaFree (both can synchronise the whole device and
// stall unrelated streams), or code that only gets a fixed memory budget at start-up.
// For them this file keeps the scratch of the apply (half spectrum, row-Nyquist
// coefficients, twiddle tables, depth nodes) in one file-scope device array of a fixed
// size, and reuses the kernels of the context-based entry point unchanged.
//
// The array lives in every device that loads the library until the process exits.
// Host code must not use the symbol's name as a device address: its device address is
// looked up with cudaGetSymbolAddress, with the caller's device current, on every call.
// The lookup is host-side and allocates nothing; it is not cached, because the address
// belongs to the current context (a cudaDeviceReset, or a caller running in a context of
// its own on the same device, loads the module again, possibly at another address).
#include <math.h>
#include <string.h>

#include "fvim_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FVIM_NOALLOC_SCRATCH_BYTES];

// device address of the scratch array in the current context
int scratch_address(void** out) {
  void* p = nullptr;
  if (FVIM_CU(cudaGetSymbolAddress(&p, g_noalloc_scratch)) || !p) return FVIM_ERR_CUDA;
  *out = p;
  return FVIM_OK;
}

// depth nodes passed by value as a kernel argument (4 KB at most), so that no host-to-device
// copy from the caller's pageable array is needed
constexpr int kMaxNodes = 512;
struct Nodes {
  double z[kMaxNodes];
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// twiddles exp(-2 pi i k / n), computed on the device in double precision
template <typename T> __global__ void k_twiddles(typename Cx<T>::t* tw, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)n, &s, &c);
  tw[k] = mk<typename Cx<T>::t>((T)c, (T)s);
}

template <typename T> __global__ void k_nodes(T* zd, const __grid_constant__ Nodes zs, int nz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nz) zd[i] = (T)zs.z[i];
}

template <typename T>
int run(fvim_ctx* c, unsigned char* base, const T* eps_p, T* out, int kind, T* u3) {
  typedef typename Cx<T>::t V;
  const int n1 = c->n1, n2 = c->n2, nz = c->nz;
  // layout of the scratch: depth nodes, twiddles, spectrum, Nyquist rows, surface spectrum;
  // every region is written before it is read, nothing needs zeroing
  size_t off = 0;
  c->z_dev = base + off;
  off += align256((size_t)nz * sizeof(T));
  c->tw1 = base + off;
  off += align256((size_t)n1 * sizeof(V));
  c->tw2 = base + off;
  off += align256((size_t)n2 * sizeof(V));
  c->spec = base + off;
  off += align256((size_t)nz * 6 * n2 * c->h1 * sizeof(V));
  c->nq = base + off;
  off += align256((size_t)nz * 6 * n2 * sizeof(T));
  c->surf = base + off;
  off += align256((size_t)n2 * c->h1 * sizeof(V));
  c->surf_nq = base + off;
  off += align256((size_t)n2 * sizeof(T));
  if (off > (size_t)FVIM_NOALLOC_SCRATCH_BYTES) return FVIM_ERR_UNSUPPORTED;
  Nodes zn;
  memset(&zn, 0, sizeof(zn));
  memcpy(zn.z, c->z_host, (size_t)nz * sizeof(double));
  k_nodes<T><<<(nz + 127) / 128, 128, 0, c->stream>>>((T*)c->z_dev, zn, nz);
  k_twiddles<T><<<(n1 + 127) / 128, 128, 0, c->stream>>>((V*)c->tw1, n1);
  k_twiddles<T><<<(n2 + 127) / 128, 128, 0, c->stream>>>((V*)c->tw2, n2);
  FVIM_CUDA_CHECK_LAUNCH();
  int rc;
  if ((rc = launch_rows_fwd6<T>(c, eps_p, 0, nz))) return rc;
  if ((rc = launch_cols<T>(c, false, c->spec, nz * 6))) return rc;
  if ((rc = launch_mindlin_depth<T>(c, kind, u3 != nullptr))) return rc;
  if ((rc = launch_cols<T>(c, true, c->spec, nz * 6))) return rc;
  if ((rc = launch_rows_inv6<T>(c, out, kind == FVIM_STRESS ? -(T)n2 : (T)0, 0, nz))) return rc;
  if (u3) {
    if ((rc = launch_cols<T>(c, true, c->surf, 1))) return rc;
    if ((rc = launch_rows_inv1<T>(c, u3))) return rc;
  }
  return FVIM_OK;
}

bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

}  // namespace

extern "C" int fvim_apply_mindlin_noalloc(int n1, int n2, int nz, const double* z_nodes, double L1, double L2,
                                          double E, double nu, int precision, const void* eps_p, void* out,
                                          int out_kind, void* u3_surface, void* stream) {
  if (!pow2(n1) || !pow2(n2) || n1 < 4 || n2 < 2 || n1 > 1024 || n2 > 1024) return FVIM_ERR_ARG;
  if (nz < 2 || nz > kMaxNodes || !z_nodes || !(L1 > 0) || !(L2 > 0)) return FVIM_ERR_ARG;
  if (precision != FVIM_FP32 && precision != FVIM_FP64) return FVIM_ERR_ARG;
  if (!(E > 0) || !(nu > -1.0 && nu < 0.5)) return FVIM_ERR_ARG;
  if (!eps_p || !out || eps_p == out) return FVIM_ERR_ARG;
  if (out_kind != FVIM_STRESS && out_kind != FVIM_STRAIN) return FVIM_ERR_ARG;
  if (z_nodes[0] != 0.0) return FVIM_ERR_ARG;
  for (int i = 1; i < nz; ++i)
    if (!(z_nodes[i] > z_nodes[i - 1]) || !isfinite(z_nodes[i])) return FVIM_ERR_ARG;
  // size check before any device work
  const size_t es = precision == FVIM_FP64 ? 8 : 4, cs = 2 * es;
  const size_t h1 = (size_t)n1 / 2;
  const size_t need = align256((size_t)nz * es) + align256((size_t)n1 * cs) +
                      align256((size_t)n2 * cs) + align256((size_t)nz * 6 * n2 * h1 * cs) +
                      align256((size_t)nz * 6 * n2 * es) + align256((size_t)n2 * h1 * cs) +
                      align256((size_t)n2 * es);
  if (need > (size_t)FVIM_NOALLOC_SCRATCH_BYTES) return FVIM_ERR_UNSUPPORTED;
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  fvim_ctx c;
  memset(&c, 0, sizeof(c));
  c.n1 = n1;
  c.n2 = n2;
  c.nz = nz;
  c.h1 = n1 / 2;
  c.hs = c.h1;
  c.fft_path = FVIM_FFT_ROWCOL;
  c.prec = precision;
  c.L1 = L1;
  c.L2 = L2;
  c.E = E;
  c.nu = nu;
  c.mu = E / (2.0 * (1.0 + nu));
  c.lam = 2.0 * c.mu * nu / (1.0 - 2.0 * nu);
  c.stream = (cudaStream_t)stream;
  c.z_host = const_cast<double*>(z_nodes);
  const double h = z_nodes[1] - z_nodes[0];
  c.uniform = 1;
  for (int i = 1; i < nz; ++i)
    if (fabs((z_nodes[i] - z_nodes[i - 1]) - h) > 1e-12 * fabs(z_nodes[nz - 1])) c.uniform = 0;
  c.hz = h;
  // a grid tuned earlier in this process (fvim_autotune) runs its tuned depth tile plan, as a
  // context created for it would (host-only table lookup)
  if ((c.depth_chunk = plan_lookup(&c)) > 0) c.plan_tuned = 1;
  c.depth_ctas = plan_lookup_ctas(&c);
  c.depth_cut = FVIM_DEPTH_CUTOFF_DEFAULT;
  if (precision == FVIM_FP64)
    return run<double>(&c, (unsigned char*)base, (const double*)eps_p, (double*)out, out_kind, (double*)u3_surface);
  return run<float>(&c, (unsigned char*)base, (const float*)eps_p, (float*)out, out_kind, (float*)u3_surface);
}

// Tile-plan autotuner of the depth kernel and of the in-plane FFT path (declarations and
// contracts in include/fvim.h).
//
// The depth range of every mode is cut into chunks of C nodes, one thread per chunk, whose
// recursion carries are combined by a log-depth scan (depth.cu).  Short chunks give more
// threads and a shorter serial recursion, long chunks fewer scan rounds and fewer threads
// per tile; which one is fastest depends on the grid (small grids are latency bound, large
// ones issue bound), so it is measured: every launchable C is timed on the context's own
// stream and the fastest is kept in a process-wide table keyed by grid, precision and depth
// spacing, so later contexts of that grid start with it.  The in-plane transforms have up to
// three complete implementations (row and column kernels; one kernel per direction exchanging
// the row spectra through L2; one cluster per plane holding them in distributed shared
// memory), whose speed also depends on the plane size: whole applies with each are timed and
// the fastest is kept in the same table.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fvim_internal.cuh"

namespace {

typedef std::tuple<int, int, int, int, int> PlanKey;  // precision, n1, n2, nz, uniform

struct PlanVal {
  int depth_chunk;
  int depth_ctas;
  int fft_path;
};

std::mutex g_plan_mu;
std::map<PlanKey, PlanVal>& plan_table() {
  static std::map<PlanKey, PlanVal> t;
  return t;
}

PlanKey key_of(const fvim_ctx* c) { return PlanKey(c->prec, c->n1, c->n2, c->nz, c->uniform); }

// candidate launch shapes (chunk length, CTAs per SM): the instantiated register-variant
// lengths, two longer ones and the default rule, each with the default register budget, then
// the lengths that also build for three CTAs per SM
struct Cand {
  int C, ctas;
  bool operator==(const Cand& o) const { return C == o.C && ctas == o.ctas; }
};
std::vector<Cand> candidates(const fvim_ctx* c) {
  std::vector<Cand> v;
  const int base[] = {2, 3, 4, 6, 8, 12, 16, depth_chunk_default(c->nz)};
  for (int ctas : {2, 3})
    for (int C : base) {
      const Cand k{C, ctas};
      if (depth_chunk_ok(c, C, ctas) && std::find(v.begin(), v.end(), k) == v.end()) v.push_back(k);
    }
  if ((int)v.size() > FVIM_PLAN_MAX_CAND) v.resize(FVIM_PLAN_MAX_CAND);
  return v;
}

int launch_depth(const fvim_ctx* c) {
  return c->prec == FVIM_FP64 ? launch_mindlin_depth<double>(c, FVIM_STRESS, false)
                              : launch_mindlin_depth<float>(c, FVIM_STRESS, false);
}

// median of reps launch times of the depth kernel with launch shape k (ms), or < 0 on error
float time_chunk(fvim_ctx* c, Cand k, int reps, std::vector<cudaEvent_t>& ev) {
  c->depth_chunk = k.C;
  c->depth_ctas = k.ctas;
  for (int w = 0; w < 2; ++w)
    if (launch_depth(c)) return -1.f;
  for (int r = 0; r < reps; ++r) {
    if (FVIM_CU(cudaEventRecord(ev[r], c->stream))) return -1.f;
    if (launch_depth(c)) return -1.f;
  }
  if (FVIM_CU(cudaEventRecord(ev[reps], c->stream))) return -1.f;
  if (FVIM_CU(cudaEventSynchronize(ev[reps]))) return -1.f;
  std::vector<float> t(reps);
  for (int r = 0; r < reps; ++r)
    if (FVIM_CU(cudaEventElapsedTime(&t[r], ev[r], ev[r + 1]))) return -1.f;
  std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
  return t[reps / 2];
}

// median of reps times of one whole Mindlin apply (stress output) with FFT path `path`, reading
// in and writing out (ms), or < 0 on error
float time_apply(fvim_ctx* c, int path, const void* in, void* out, int reps, std::vector<cudaEvent_t>& ev) {
  c->fft_path = path;
  auto apply = [&] {
    return c->prec == FVIM_FP64
               ? apply_mindlin_t<double>(c, (const double*)in, (double*)out, FVIM_STRESS, nullptr)
               : apply_mindlin_t<float>(c, (const float*)in, (float*)out, FVIM_STRESS, nullptr);
  };
  for (int w = 0; w < 2; ++w)
    if (apply()) return -1.f;
  for (int r = 0; r < reps; ++r) {
    if (FVIM_CU(cudaEventRecord(ev[r], c->stream))) return -1.f;
    if (apply()) return -1.f;
  }
  if (FVIM_CU(cudaEventRecord(ev[reps], c->stream))) return -1.f;
  if (FVIM_CU(cudaEventSynchronize(ev[reps]))) return -1.f;
  std::vector<float> t(reps);
  for (int r = 0; r < reps; ++r)
    if (FVIM_CU(cudaEventElapsedTime(&t[r], ev[r], ev[r + 1]))) return -1.f;
  std::nth_element(t.begin(), t.begin() + reps / 2, t.end());
  return t[reps / 2];
}

void fill_plan(const fvim_ctx* c, fvim_plan* out) {
  out->depth_chunk = c->depth_chunk > 0 ? c->depth_chunk : depth_chunk_default(c->nz);
  out->tuned = c->plan_tuned;
  out->depth_ctas = depth_launch_ctas(c);
  out->depth_cutoff = c->depth_cut;
  out->fft_path = c->fft_path >= 0 ? c->fft_path : FVIM_FFT_ROWCOL;
}

}  // namespace

int plan_lookup(const fvim_ctx* c) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = plan_table().find(key_of(c));
  return it == plan_table().end() ? 0 : it->second.depth_chunk;
}

int plan_lookup_fft(const fvim_ctx* c) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = plan_table().find(key_of(c));
  return it == plan_table().end() ? -1 : it->second.fft_path;
}

int plan_lookup_ctas(const fvim_ctx* c) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = plan_table().find(key_of(c));
  return it == plan_table().end() ? 0 : it->second.depth_ctas;
}

extern "C" {

int fvim_autotune(fvim_ctx* c, int reps, fvim_plan* out) {
  if (!c || reps < 1 || reps > 1000) return FVIM_ERR_ARG;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (FVIM_CU(cudaStreamIsCapturing(c->stream, &cs))) return FVIM_ERR_CUDA;
  if (cs != cudaStreamCaptureStatusNone) return FVIM_ERR_ARG;
  const std::vector<Cand> cand = candidates(c);
  if (cand.empty()) return FVIM_ERR_UNSUPPORTED;
  const int old = c->depth_chunk > 0 ? c->depth_chunk : depth_chunk_default(c->nz);
  const int old_ctas = c->depth_ctas;
  const int old_fft = c->fft_path;
  // the kernel runs in place on the context's spectrum scratch; zeros take the same path
  const size_t es = c->prec == FVIM_FP64 ? 8 : 4;
  if (FVIM_CU(cudaMemsetAsync(c->spec, 0, (size_t)c->nz * 6 * c->n2 * c->h1 * 2 * es, c->stream))) return FVIM_ERR_CUDA;
  std::vector<cudaEvent_t> ev(reps + 1, nullptr);
  int rc = FVIM_OK;
  for (auto& e : ev)
    if (FVIM_CU(cudaEventCreate(&e))) { rc = FVIM_ERR_CUDA; break; }
  std::vector<float> ms(cand.size(), -1.f);
  for (size_t i = 0; rc == FVIM_OK && i < cand.size(); ++i) {
    ms[i] = time_chunk(c, cand[i], reps, ev);
    if (ms[i] < 0) rc = FVIM_ERR_CUDA;
  }
  // the default rule keeps its place unless another length is faster by more than 2 %
  // (timing noise does not flip the plan)
  if (rc == FVIM_OK) {
    const Cand def{depth_chunk_default(c->nz), 2};
    size_t best = 0;
    for (size_t i = 1; i < cand.size(); ++i)
      if (ms[i] < ms[best]) best = i;
    for (size_t i = 0; i < cand.size(); ++i)
      if (cand[i] == def && ms[best] > 0.98f * ms[i]) best = i;
    c->depth_chunk = cand[best].C;
    c->depth_ctas = cand[best].ctas;
  }
  // then the in-plane FFT path, timed on whole applies with that chunk length (the row / column
  // path unless another is more than 2 % faster)
  float fms[FVIM_FFT_NPATH] = {0.f, 0.f, 0.f};
  int npaths = 0;
  for (int f = 0; f < FVIM_FFT_NPATH; ++f) npaths += fft_path_available(c, f) ? 1 : 0;
  int best_fft = FVIM_FFT_ROWCOL;
  if (rc == FVIM_OK && npaths > 1) {
    void* tmp = nullptr;
    if (FVIM_CU(cudaMalloc(&tmp, (size_t)c->nz * 6 * c->n2 * c->n1 * es))) {
      cudaGetLastError();
      rc = FVIM_ERR_OOM;
    }
    for (int f = 0; rc == FVIM_OK && f < FVIM_FFT_NPATH; ++f) {
      if (!fft_path_available(c, f)) continue;
      fms[f] = time_apply(c, f, c->st_eps_p, tmp, reps, ev);
      if (fms[f] < 0) rc = FVIM_ERR_CUDA;
    }
    if (tmp) {
      cudaStreamSynchronize(c->stream);
      cudaFree(tmp);
    }
    for (int f = 1; rc == FVIM_OK && f < FVIM_FFT_NPATH; ++f)
      if (fms[f] > 0 && fms[f] < 0.98f * fms[best_fft] && (best_fft == FVIM_FFT_ROWCOL || fms[f] < fms[best_fft]))
        best_fft = f;
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (rc) {
    c->depth_chunk = old;
    c->depth_ctas = old_ctas;
    c->fft_path = old_fft;
    return rc;
  }
  c->fft_path = best_fft;
  c->plan_tuned = 1;
  // captured graphs hold the old launch shapes and kernels
  if (c->depth_chunk != old || c->depth_ctas != old_ctas || c->fft_path != old_fft) solver_drop_graphs(c);
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    plan_table()[key_of(c)] = PlanVal{c->depth_chunk, c->depth_ctas, c->fft_path};
  }
  if (out) {
    memset(out, 0, sizeof(*out));
    fill_plan(c, out);
    out->n_cand = (int)cand.size();
    for (size_t i = 0; i < cand.size(); ++i) {
      out->cand[i] = cand[i].C;
      out->cand_ctas[i] = cand[i].ctas;
      out->cand_ms[i] = ms[i];
    }
    for (int f = 0; f < FVIM_FFT_NPATH; ++f) out->fft_ms[f] = fms[f];
  }
  return FVIM_OK;
}

int fvim_plan_candidates(int n1, int n2, int nz, int precision, int* chunks, int* ctas, int max_chunks) {
  if (!grid_ok(n1, n2) || nz < 2 || nz > 512) return FVIM_ERR_ARG;
  if ((precision != FVIM_FP32 && precision != FVIM_FP64) || !chunks || max_chunks < 1) return FVIM_ERR_ARG;
  // the launch rules need the grid and precision only: a host-side description of the grid
  fvim_ctx g;
  memset(&g, 0, sizeof(g));
  g.n1 = n1;
  g.n2 = n2;
  g.nz = nz;
  g.gen = grid_gen(n1, n2) ? 1 : 0;
  g.h1 = spec_stride(n1, n2);
  g.hs = g.gen ? n1 / 2 + 1 : g.h1;
  g.prec = precision;
  const std::vector<Cand> cand = candidates(&g);
  const int n = (int)cand.size() < max_chunks ? (int)cand.size() : max_chunks;
  for (int i = 0; i < n; ++i) {
    chunks[i] = cand[i].C;
    if (ctas) {
      g.depth_chunk = cand[i].C;
      g.depth_ctas = cand[i].ctas;
      ctas[i] = depth_launch_ctas(&g);
    }
  }
  return n;
}

int fvim_get_plan(const fvim_ctx* c, fvim_plan* out) {
  if (!c || !out) return FVIM_ERR_ARG;
  memset(out, 0, sizeof(*out));
  fill_plan(c, out);
  return FVIM_OK;
}

int fvim_set_plan(fvim_ctx* c, const fvim_plan* plan) {
  if (!c || !plan) return FVIM_ERR_ARG;
  const int C = plan->depth_chunk;
  const int ctas = plan->depth_ctas == 3 ? 3 : 2;
  if (plan->depth_ctas != 0 && plan->depth_ctas != 2 && plan->depth_ctas != 3) return FVIM_ERR_ARG;
  if (!(plan->depth_cutoff >= 0.f) || !(plan->depth_cutoff < 1e30f)) return FVIM_ERR_ARG;
  if (!depth_chunk_ok(c, C > 0 ? C : depth_chunk_default(c->nz), ctas)) return FVIM_ERR_ARG;
  if (plan->fft_path < 0 || plan->fft_path >= FVIM_FFT_NPATH || !fft_path_available(c, plan->fft_path))
    return FVIM_ERR_ARG;
  const int old = c->depth_chunk > 0 ? c->depth_chunk : depth_chunk_default(c->nz);
  const int old_ctas = c->depth_ctas, old_fft = c->fft_path;
  const float old_cut = c->depth_cut;
  c->depth_chunk = C;
  c->depth_ctas = ctas;
  c->depth_cut = plan->depth_cutoff;
  c->fft_path = plan->fft_path;
  c->plan_tuned = 0;
  if ((C > 0 ? C : depth_chunk_default(c->nz)) != old || c->depth_ctas != old_ctas || c->fft_path != old_fft ||
      c->depth_cut != old_cut)
    solver_drop_graphs(c);
  return FVIM_OK;
}

}  // extern "C"

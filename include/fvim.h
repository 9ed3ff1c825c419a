/*
 * fvim.h -- C ABI of the GB300 (sm_103a) implementation of the Fourier-accelerated
 * volume integral method for elastoplastic contact (Frerot, Bonnet, Molinari &
 * Anciaux, arXiv:1811.11558).
 *
 * Problem (Sec. 1): a horizontally periodic half-space y3 >= 0 (e3 points into the
 * body), periodic cell ]-L1/2, L1/2[ x ]-L2/2, L2/2[ (Eq. periodic_cell), discretised
 * on N1 x N2 in-plane points and Nz depth nodes X3 = {z_0 = 0 < z_1 < ... < z_{Nz-1}}
 * (Sec. 3.1).  Isotropic elasticity (E, nu), J2 plasticity with linear isotropic
 * hardening (sigma_y, E_h) (Sec. 4.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Symmetric tensors are stored as six TENSOR components in the order
 *   (11, 22, 33, 23, 13, 12); shears are eps_ij, not engineering shears.
 * - Volume fields are contiguous [Nz][6][N2][N1] arrays (x1 fastest); surface fields
 *   are contiguous [N2][N1]; scalar volume fields are [Nz][N2][N1].
 * - Element type is float for FVIM_FP32 contexts and double for FVIM_FP64 contexts.
 * - Pointers marked "device" are CUDA device pointers owned by the caller; the library
 *   never frees them.  The context owns its scratch buffers and its plastic state.
 * - Every call is enqueued on the context's CUDA stream and returns before the GPU has
 *   finished (stream ordered), unless stated otherwise.  Arguments are checked on the
 *   host before anything is launched.  Functions never throw across the ABI; they
 *   return FVIM_OK or a negative status.
 * - Pressure p >= 0 pushes into the body (a force p e3 per unit area, Sec. 1.1),
 *   so sigma_33 = -p on the surface; u3 > 0 is a displacement into the body.
 * - A context is used by one host thread at a time; different contexts may be used from
 *   different threads at once (each solver call runs on the context's own stream).
 */
#ifndef FVIM_H
#define FVIM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FVIM_FP32 0
#define FVIM_FP64 1

#define FVIM_STRESS 0 /* output sigma = C:grad^sym N[w] - w (or C:grad^sym M[p]) */
#define FVIM_STRAIN 1 /* output grad^sym N[w] (or grad^sym M[p])                 */

enum {
  FVIM_OK = 0,
  FVIM_ERR_ARG = -1,           /* invalid argument (size, pointer, kind)          */
  FVIM_ERR_OOM = -2,           /* device allocation failed                         */
  FVIM_ERR_CUDA = -3,          /* a CUDA runtime call or launch failed             */
  FVIM_ERR_NONFINITE = -4,     /* non-finite value detected                        */
  FVIM_ERR_NOT_CONVERGED = -5, /* iteration cap reached before the tolerance       */
  FVIM_ERR_TIMEOUT = -6,       /* bounded device wait expired                      */
  FVIM_ERR_UNSUPPORTED = -7    /* valid request the library does not support      */
};

typedef struct fvim_ctx fvim_ctx;

/*
 * fvim_create -- grid, depth nodes, periodic cell and precision (Sec. 3.1, Eq.
 * periodic_cell).
 *   out        receives the new context (host pointer to an opaque handle).
 *   n1, n2     in-plane points: powers of two, 4 <= n1 <= 1024, 2 <= n2 <= 1024 (FFTs), or
 *              a grid with an odd side 3..255 whose other side is odd (3..255) or a power
 *              of two up to 256 (direct DFTs of Sec. 3.1, e.g. 81 x 81 of App. C.2).  On
 *              an odd side every mode is in Z^2_N; on an even side the Nyquist mode
 *              k = N/2 carries no operator term.
 *   nz         depth nodes, 2 <= nz <= 512.
 *   z_nodes    HOST array of nz depths, z_nodes[0] == 0, strictly increasing.
 *   L1, L2     cell lengths (> 0).
 *   precision  FVIM_FP32 or FVIM_FP64: element type of every array argument.
 *   stream     cudaStream_t to enqueue on (NULL = legacy default stream).
 * The context allocates its scratch on the current CUDA device (FVIM_ERR_OOM if
 * that fails).  Material defaults: E = 1, nu = 0.3, sigma_y = inf, E_h = 0.  A grid
 * whose depth-kernel tile plan was tuned earlier in this process (fvim_autotune) starts
 * with that plan.
 */
int fvim_create(fvim_ctx** out, int n1, int n2, int nz, const double* z_nodes,
                double L1, double L2, int precision, void* stream);

/* fvim_set_material -- isotropic C(E, nu) and linear hardening f_h = sigma_y + E_h e_p
 * (Sec. 4.1).  E > 0, -1 < nu < 0.5, sigma_y > 0, E_h >= 0. */
int fvim_set_material(fvim_ctx* ctx, double E, double nu, double sigma_y, double E_h);

/* fvim_set_stream -- change the stream later calls are enqueued on. */
int fvim_set_stream(fvim_ctx* ctx, void* stream);

/*
 * fvim_apply_mindlin -- the Mindlin operator (Eq. N:conv, Thm 1, Eq. 2gradient,
 * Eq. jump, Eq. mindlin_B_U) applied to the eigenstress w = C:eps_p.
 *   eps_p       device, [Nz][6][N2][N1], plastic strain (input, not modified).
 *   out         device, [Nz][6][N2][N1]: sigma = C:grad^sym N[w] - w (FVIM_STRESS,
 *               Sec. 6.1) or grad^sym N[w] (FVIM_STRAIN).  May not alias eps_p.
 *   out_kind    FVIM_STRESS or FVIM_STRAIN.
 *   u3_surface  device [N2][N1] or NULL: surface normal displacement N[w].e3 at z = 0
 *               (mode k = 0 set to zero, Rem. fundamental_mode).
 * Modes k1 = N1/2 or k2 = N2/2 (not in Z^2_N, Sec. 3.1) carry no operator term.
 */
int fvim_apply_mindlin(fvim_ctx* ctx, const void* eps_p, void* out, int out_kind, void* u3_surface);

/*
 * fvim_apply_mindlin_group -- fvim_apply_mindlin on n independent problems of uneven grid
 * size in one launch per pass: forward rows, forward columns, depth operator, inverse
 * columns, inverse rows, five launches for the whole group (the operator of Thm 1 per
 * problem, Sec. 3.1-3.2; batching many surfaces has no counterpart in the paper, which
 * solves one problem at a time).  Every CTA of a launch looks its problem up in a table that
 * travels as a kernel parameter, so the call allocates nothing, copies nothing to the device
 * and can be captured in a CUDA graph.
 *   ctx        HOST array of n distinct FP32 contexts whose grids have power-of-two sides
 *              64 <= N1, N2 <= 512 and 4 <= Nz <= 64; problem i uses ctx[i]'s grid,
 *              material and scratch buffers.
 *   eps_p, out HOST arrays of n device pointers, each as for fvim_apply_mindlin (out may
 *              not alias eps_p).  No surface displacement output.
 *   out_kind   FVIM_STRESS or FVIM_STRAIN, for every problem.
 *   stream     cudaStream_t the launches go to (NULL = legacy default stream).  The
 *              contexts' scratch buffers are shared with their own calls: the caller orders
 *              the group after any work of those contexts on their own streams.
 * Problem i gives the result of fvim_apply_mindlin(ctx[i], eps_p[i], out[i], out_kind,
 * NULL) under the depth plan {chunk length 4, the context's cutoff}, except that the cutoff
 * of Sec. 3.2 is decided for the tiles a CTA holds together (with cutoff 0 the results are
 * bitwise the same).  1 <= n <= FVIM_GROUP_MAX.  Returns FVIM_ERR_ARG for bad arguments
 * (n out of range, a NULL or repeated context or pointer) and FVIM_ERR_UNSUPPORTED for a
 * context outside the shapes above; nothing is launched then.
 */
#define FVIM_GROUP_MAX 64
int fvim_apply_mindlin_group(fvim_ctx* const* ctx, int n, const void* const* eps_p, void* const* out, int out_kind,
                             void* stream);

/*
 * fvim_apply_boussinesq -- the Boussinesq operator M[p] for a normal surface pressure
 * (Eq. M:conv, Eq. B:fourier).
 *   p           device [N2][N1] pressure (input).
 *   u3_surface  device [N2][N1] or NULL: u3 = M[p].e3 at z = 0, u3_hat = 2 p_hat/(E* q),
 *               mode 0 set to zero.
 *   vol_out     device [Nz][6][N2][N1] or NULL: C:grad^sym M[p] (FVIM_STRESS) or
 *               grad^sym M[p] (FVIM_STRAIN) at every node.
 */
int fvim_apply_boussinesq(fvim_ctx* ctx, const void* p, void* u3_surface, void* vol_out, int out_kind);

/*
 * fvim_return_map -- J2 radial return with linear isotropic hardening (Sec. 4.1) for
 * a strain increment, from the context's plastic state (sigma_n, e_p).  The state is
 * read, not updated (fvim_commit_state updates it).
 *   d_eps    device [Nz][6][N2][N1] total strain increment (input).
 *   d_eps_p  device [Nz][6][N2][N1] plastic strain increment (output).
 *   d_ep     device [Nz][N2][N1] increment of cumulated plastic strain (output) or NULL.
 */
int fvim_return_map(fvim_ctx* ctx, const void* d_eps, void* d_eps_p, void* d_ep);

/* fvim_commit_state -- S_{n+1} = S_n + increment: sigma_n += C:(d_eps - d_eps_p),
 * e_p += d_ep (Sec. 4.2 update(S)).  d_eps, d_eps_p: [Nz][6][N2][N1]; d_ep: [Nz][N2][N1]. */
int fvim_commit_state(fvim_ctx* ctx, const void* d_eps, const void* d_eps_p, const void* d_ep);

/* fvim_get_state / fvim_set_state -- device-to-device copies of the plastic state S_n of
 * Sec. 4.2 (the state S that Algorithm 1 of Sec. 5.2 updates after each converged
 * increment): eps_p [Nz][6][N2][N1] (accumulated plastic strain), e_p [Nz][N2][N1]
 * (cumulated plastic strain of the hardening law, Sec. 4.1), and sigma [Nz][6][N2][N1],
 * the stress of the last converged increment that the trial stress of the return map
 * starts from.  Any pointer may be NULL to skip that field. */
int fvim_get_state(fvim_ctx* ctx, void* eps_p, void* e_p, void* sigma);
int fvim_set_state(fvim_ctx* ctx, const void* eps_p, const void* e_p, const void* sigma);

/* fvim_reset_state -- virgin state S_0 of Algorithm 1 (Sec. 5.2): eps_p = 0, e_p = 0,
 * sigma = 0 and no contact pressure (stream ordered).  Lets one context serve a sequence
 * of independent problems. */
int fvim_reset_state(fvim_ctx* ctx);

/* fvim_footprint -- device bytes a context of this grid and precision holds once its
 * solvers have run (scratch, plastic state and solver workspace); host computation only. */
size_t fvim_footprint(int n1, int n2, int nz, int precision);

/* fvim_sync -- wait for the context's stream; returns FVIM_ERR_CUDA on a device error and
 * FVIM_ERR_TIMEOUT (once; the status is then cleared) when a bounded wait inside a kernel
 * launched since the last fvim_sync expired (the kernel returned without its output: the
 * results of those calls are invalid). */
int fvim_sync(fvim_ctx* ctx);

/* fvim_destroy -- free the context and its scratch (synchronises its stream). */
int fvim_destroy(fvim_ctx* ctx);

/* fvim_strerror -- static description of a status code. */
const char* fvim_strerror(int status);

/* fvim_last_cuda_error -- description of the last CUDA runtime error that made an entry
 * point return FVIM_ERR_CUDA (or that a solver recovered from by launching directly
 * instead of through a captured graph) in the calling host thread, followed by the source
 * file and line of the runtime call that returned it; "no error" if none.  The string is
 * owned by the library and stays valid until the thread's next failing call.  The paper
 * has no counterpart: it is the diagnostic behind FVIM_ERR_CUDA. */
const char* fvim_last_cuda_error(void);

/*
 * Tile plan of the per-wavevector depth kernel.  The paper has no counterpart: its depth
 * integral (Sec. 3.2) is evaluated here by exact O(Nz) exponential recursions whose depth
 * range is cut into chunks of depth_chunk nodes, one thread per chunk, the chunk carries
 * being combined by a log-depth scan.  Every launchable chunk length gives the same operator
 * up to the rounding order of that scan; the fastest one depends on the grid.
 *   depth_chunk   chunk length in use (fvim_set_plan: 0 selects the default rule,
 *                 max(2, ceil(Nz / 16)))
 *   tuned         1 if depth_chunk came from a timing run (fvim_autotune) in this process
 *   n_cand, cand[i], cand_ctas[i], cand_ms[i]   fvim_autotune only: the launch shapes timed
 *                 (chunk length, CTAs per SM) and the median time of one depth-kernel launch
 *                 with each (ms)
 *   depth_cutoff  eps_co of the FP32 register variant's chunk scan (the cutoff of Sec. 3.2,
 *                 restated for the exact recursion): a tile whose chunk spans all damp by
 *                 e^{-q span} < e^{-eps_co} takes each chunk's carry from its neighbour alone,
 *                 skipping the log-depth scan (the dropped terms are below e^{-eps_co} of the
 *                 moments).  Default FVIM_DEPTH_CUTOFF_DEFAULT = 18 (e^{-18} = 1.5e-8, below the
 *                 FP32 rounding unit); fvim_set_plan: 0 selects the exact scan.  Not used by
 *                 the shared-memory variant (FP64, deep grids), whose scan is sequential.
 *   depth_ctas    CTAs per SM the FP32 register variant of the depth kernel is compiled for:
 *                 2 (128 registers per thread, the default) or 3 (85 registers, chunk lengths
 *                 4..8 whose tile fits three times in shared memory); 0 for the shared-memory
 *                 variant (FP64, deep grids), which has one launch shape per chunk length
 */
#define FVIM_PLAN_MAX_CAND 16
#define FVIM_DEPTH_CUTOFF_DEFAULT 18.0f
/* in-plane FFT paths of the Mindlin apply (FP32 grids; every path gives the same operator up to
 * rounding): FVIM_FFT_ROWCOL separate row and column kernels (every grid), FVIM_FFT_L2 one
 * kernel per direction with the row spectra exchanged through L2, FVIM_FFT_CLUSTER one kernel
 * per direction with the row spectra in distributed shared memory (some plane sizes) */
#define FVIM_FFT_ROWCOL 0
#define FVIM_FFT_L2 1
#define FVIM_FFT_CLUSTER 2
#define FVIM_FFT_NPATH 3
typedef struct fvim_plan {
  int depth_chunk;
  int tuned;
  int n_cand;
  int cand[FVIM_PLAN_MAX_CAND];
  int cand_ctas[FVIM_PLAN_MAX_CAND];
  float cand_ms[FVIM_PLAN_MAX_CAND];
  int depth_ctas;
  float depth_cutoff;
  int fft_path;                    /* path in use (FVIM_FFT_*)                                   */
  float fft_ms[FVIM_FFT_NPATH];    /* fvim_autotune: median time of one whole apply with each
                                      path, in ms (0: not built for this grid or precision)      */
} fvim_plan;

/* fvim_autotune -- times the depth kernel on ctx's grid with every launchable chunk length
 * of {2, 3, 4, 6, 8, 12, 16} and the default, each with every register budget it is built
 * for (depth_ctas 2 and 3), `reps` launches each on ctx's stream over its (zeroed) spectrum
 * scratch, and keeps the fastest (the default unless another is more than 2 % faster); then, with that chunk length, times `reps` whole Mindlin applies (stress
 * output) with every in-plane FFT path built for the grid and keeps the fastest (the
 * row / column path unless another is more than 2 % faster).  The plan holds for ctx and for
 * every context of the same grid, precision and depth spacing (uniform or not) created later
 * in this process.  The apply timings read the context's plastic-strain state as input and
 * write one volume buffer that the call allocates and frees (the only allocation it makes).
 * Synchronises ctx's stream; leaves the plastic state untouched; drops ctx's captured solver
 * graphs when the plan changes.  out (host) or NULL receives the plan and the timings.
 * FVIM_ERR_ARG: NULL ctx, reps outside [1, 1000], or ctx's stream is capturing a graph;
 * FVIM_ERR_OOM if the timing buffer cannot be allocated; FVIM_ERR_CUDA on a device error
 * (the plan is then unchanged). */
int fvim_autotune(fvim_ctx* ctx, int reps, fvim_plan* out);

/* fvim_plan_candidates -- the depth-kernel launch shapes fvim_autotune would time on a grid
 * (n1, n2, nz, precision as in fvim_create), in timing order: chunk lengths in chunks[0..] and
 * the register budget of each (CTAs per SM, 2 or 3; 0 for the shared-memory variant) in
 * ctas[0..] (host arrays, at most max_chunks entries; ctas may be NULL); returns their number.
 * Host computation only (no device, no context).  FVIM_ERR_ARG on a grid fvim_create refuses
 * or a bad output array. */
int fvim_plan_candidates(int n1, int n2, int nz, int precision, int* chunks, int* ctas, int max_chunks);

/* fvim_get_plan -- the plan ctx uses (host out; cand and fft_ms fields zero). */
int fvim_get_plan(const fvim_ctx* ctx, fvim_plan* out);

/* fvim_set_plan -- forces plan->depth_chunk, plan->depth_ctas (0 or 2: the default budget),
 * plan->depth_cutoff (>= 0; 0: exact scan) and plan->fft_path on ctx alone (other fields
 * ignored); the process table is not changed.
 * FVIM_ERR_ARG if that launch shape is not launchable on ctx's grid (more than 256 chunk
 * threads per tile, the tile does not fit in shared memory, or no such register budget) or
 * that FFT path is not built for ctx's grid and precision. */
int fvim_set_plan(fvim_ctx* ctx, const fvim_plan* plan);

/* fvim_last_kernel_count -- number of kernels the last entry point launched. */
int fvim_last_kernel_count(const fvim_ctx* ctx);

/*
 * Kernel timing.  While enabled, every kernel the context launches is bracketed by
 * two CUDA events recorded on the context's stream.  fvim_profile_read synchronises
 * the stream, adds up the elapsed times per kernel kind and clears the records:
 *   total_ms[s], launches[s] for s < nslots (host arrays), slot names from
 *   fvim_profile_name(s) (NULL past the last slot).
 */
int fvim_profile_enable(fvim_ctx* ctx, int on);
int fvim_profile_read(fvim_ctx* ctx, double* total_ms, int* launches, int nslots);
const char* fvim_profile_name(int slot);

/* ------------------------------------------------------------------------------------
 * Solvers.  Vectors live on the device in the context's precision; every reduction
 * (dot products, norms, the total load) is accumulated in FP64 in a fixed order (block
 * partials summed in block order by the last block to finish), so repeated runs give
 * bitwise identical results.  The iteration logic runs on the device: the contact CG's
 * scalars (step, conjugation, rigid shift, load scaling, stop test) are kept in device
 * memory; the CG iterations and DF-SANE's iterations with its line search each run inside
 * one captured CUDA graph (a device-side WHILE loop), and the host reads their state once
 * per solve (batches of captured CG iterations with one status read per batch when
 * FVIM_DEVICE_CG=0).  Every loop has an iteration cap, enforced on the device.
 * ------------------------------------------------------------------------------------ */
#define FVIM_MAX_INCREMENTS 64

typedef struct {
  double tol;         /* Algorithm 1: e = ||dU - dU_prev|| / ||H0|| < tol (paper: 1e-9)     */
  int max_iter;       /* Algorithm 1: N_max                                                  */
  double relax;       /* Algorithm 1: relaxation lambda in ]0, 1]                           */
  double cg_tol;      /* contact: dA sum |p - p_prev| / W < cg_tol                            */
  int cg_max_iter;
  double df_tol_abs;  /* DF-SANE: ||R|| <= df_tol_abs + df_tol_rel ||R_0|| (discrete L2 norm) */
  double df_tol_rel;
  int df_max_iter;
  int relax_mode;     /* Algorithm 1's relaxation: FVIM_RELAX_LITERAL or FVIM_RELAX_CARRIED          */
} fvim_opts;

/* Algorithm 1 (Sec. 5.2) relaxes dU_prev <- dU_prev + lambda (dU - dU_prev), sets H = H0 - dU_prev
 * and then overwrites dU_prev <- dU.  FVIM_RELAX_LITERAL keeps that order (the next H blends the
 * last two raw iterates; e compares raw iterates).  FVIM_RELAX_CARRIED skips the overwrite, so
 * the relaxed value is carried from iteration to iteration (under-relaxation of the fixed point
 * dU = F(H0 - dU); e = ||dU - relaxed|| / ||H0||, the fixed-point residual), the behaviour the
 * paper's text ascribes to lambda ("helps the algorithm to converge on large loading steps"):
 * with the literal order a strongly coupled increment converges only if its coupling gain a
 * satisfies a (1 - lambda) < 1, so a smaller lambda does not help; carried, any a converges for a
 * small enough lambda.  Both have the same converged increments. */
#define FVIM_RELAX_LITERAL 0
#define FVIM_RELAX_CARRIED 1

typedef struct {
  int status;                                  /* FVIM_OK or FVIM_ERR_NOT_CONVERGED        */
  int n_increments;                            /* increments completed                      */
  int alg1_iters[FVIM_MAX_INCREMENTS];         /* Algorithm-1 iterations per increment      */
  double alg1_error[FVIM_MAX_INCREMENTS];      /* final e per increment                     */
  double contact_area[FVIM_MAX_INCREMENTS];    /* fraction of surface points with p > 0     */
  double load_error;                           /* max |dA sum p - W| / W over increments    */
  long cg_iters;                               /* total contact CG iterations               */
  long df_iters;                               /* total DF-SANE iterations                  */
  long residual_evals;                         /* total plastic-residual evaluations        */
  long mindlin_applies;                        /* total Mindlin-operator applies            */
} fvim_report;

/* fvim_default_opts -- the defaults: tol 1e-9 (FP64) / 1e-8 (FP32), max_iter 100, relax 1,
 * cg_tol 1e-12 / 1e-7, cg_max_iter 2000, df_tol_abs 0, df_tol_rel 1e-10 / 1e-6,
 * df_max_iter 500, relax_mode FVIM_RELAX_LITERAL. */
int fvim_default_opts(const fvim_ctx* ctx, fvim_opts* opts);

/*
 * fvim_elastic_contact -- elastic normal contact with the rigid surface h under the total
 * load W (Sec. 5.1; constrained conjugate gradient of Polonsky & Keer 1999 on the dual
 * problem, u3 = K*p with K_hat = 2/(E* q)).
 *   h     device [N2][N1] surface profile (the rigid surface is z = h, e3 into the body).
 *   p     device [N2][N1]: initial guess on entry (all zero = uniform W/(L1 L2)), contact
 *         pressure on exit (p >= 0, dA sum p = W).
 *   iters, err: host outputs (may be NULL).  FVIM_ERR_NOT_CONVERGED at cg_max_iter.
 */
int fvim_elastic_contact(fvim_ctx* ctx, const void* h, double W, void* p, const fvim_opts* opts,
                         int* iters, double* err);

/*
 * fvim_plasticity_solve -- DF-SANE solve (Sec. 4.3) of the implicit incremental equation
 *   R[dE] = dE - grad^sym M[dT] - grad^sym N[C:deps_p(dE; S_n)] = 0   (Sec. 4.2)
 * for a surface pressure increment dT, from the context's state S_n (not updated).
 *   dT     device [N2][N1];  dE device [Nz][6][N2][N1] (output, strain increment);
 *   deps_p device [Nz][6][N2][N1] or NULL, dep device [Nz][N2][N1] or NULL: the return
 *          map of dE.  iters, res: host outputs (may be NULL).
 */
int fvim_plasticity_solve(fvim_ctx* ctx, const void* dT, void* dE, void* deps_p, void* dep,
                          const fvim_opts* opts, int* iters, double* res);

/*
 * fvim_solve_contact -- elastic-plastic contact, Algorithm 1 of Sec. 5.2, for n_inc load
 * increments loads[0..n_inc-1] (HOST array, total loads W), from the context's state.
 *   h      device [N2][N1] surface profile.
 *   p_out  device [N2][N1] contact pressure after the last increment (or NULL).
 *   rep    host report (may be NULL).
 * The plastic state (eps_p, e_p, sigma) and the last pressure are updated in the context
 * after each converged increment.  Synchronises the stream.  Returns
 * FVIM_ERR_NOT_CONVERGED if an increment reaches max_iter (the state is still updated).
 */
int fvim_solve_contact(fvim_ctx* ctx, const void* h, const double* loads, int n_inc,
                       const fvim_opts* opts, void* p_out, fvim_report* rep);

/*
 * fvim_apply_mindlin_noalloc -- the Mindlin apply of fvim_apply_mindlin without a
 * context and without any device allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory while they run (a host
 * framework that owns all device memory through its own pool, a service that must
 * never reach cudaMalloc/cudaFree because they can synchronise the whole device, or
 * code with a fixed memory budget decided at start-up).
 *
 * Its scratch (half spectrum, row-Nyquist coefficients, twiddles, depth nodes) lives in
 * one static device array of FVIM_NOALLOC_SCRATCH_BYTES bytes inside the library; every
 * GPU that loads the library holds that array until the process exits.  The caller
 * still owns the input and output buffers.
 *   n1, n2, nz, z_nodes (HOST), L1, L2, precision: as for fvim_create.
 *   E, nu: isotropic elasticity as for fvim_set_material.
 *   eps_p, out, out_kind, u3_surface: as for fvim_apply_mindlin (device buffers).
 *   stream: cudaStream_t to enqueue on (NULL = legacy default stream).
 * Returns FVIM_ERR_UNSUPPORTED, before any device work, when the scratch the grid needs
 * exceeds FVIM_NOALLOC_SCRATCH_BYTES (e.g. 128 x 128 x 32 fits in FP32, 512 x 512 x 64
 * does not).  It never calls cudaMalloc, cudaFree or any allocating routine.
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress, a host-side lookup that allocates nothing), so a device reset or
 * a caller's own context never sees a stale address.  The first call on a device may load
 * the library's device code there: make that first call before any stream capture.
 * The depth nodes travel as a kernel argument (no host-to-device copy), and a grid tuned
 * earlier in the process (fvim_autotune) runs its tuned depth tile plan.
 * Every call shares the one array and leaves its contents behind (each call overwrites
 * every region before reading it, so nothing has to be cleared): two calls that overlap
 * on the GPU (different streams, or different host threads on one device) race on it.
 */
#define FVIM_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int fvim_apply_mindlin_noalloc(int n1, int n2, int nz, const double* z_nodes, double L1, double L2,
                               double E, double nu, int precision, const void* eps_p, void* out,
                               int out_kind, void* u3_surface, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FVIM_H */

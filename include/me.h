/*
 * me.h -- C ABI of the GB300 tree-level matrix-element engine.
 *
 * The library evaluates, for every phase-space point of a Standard Model
 * tree-level process, the spin- and colour-summed squared amplitude averaged
 * over the initial helicities and colours,
 *
 *     |M|^2 = 1/(4 n_a n_b) sum_lambda sum_c | sum_diagrams M |^2
 *
 * (Hagiwara, Kanzaki, Li, Okamura, Stelzer, arXiv:1305.0708, Sect. 2,
 * Eqs. 4-6), and the Monte Carlo estimate of the partonic cross section
 * d sigma-hat = 1/(2 s-hat) |M|^2 dPhi_n (Eqs. 4-5) over on-device phase-space
 * points with cuts.  Processes are compiled ahead of time by the package's
 * process compiler (the converter of Sect. 5) and selected by name.
 *
 * Conventions for every entry point:
 *  - Return value: ME_OK (0) or a negative me_status; me_last_error() gives a
 *    thread-local description of the last failure.  Argument errors are
 *    detected before any device work is queued.
 *  - Pointers named "device" must be device-accessible memory of the current
 *    CUDA device; "host" pointers are host memory.  The caller owns every
 *    buffer it passes; the library owns the handle, its device-resident
 *    program data and its workspace.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    queued on it asynchronously unless the entry point says it synchronises.
 *  - Momenta are FP64 four-vectors (E, px, py, pz) in GeV, metric (+,-,-,-),
 *    stored structure-of-arrays: component mu of leg k of event i is at
 *    momenta[(k * 4 + mu) * n + i].  Incoming partons come first and carry
 *    physical (positive-energy) momenta; legs follow the process string.
 *  - A handle is immutable after me_create: concurrent calls on different
 *    streams are allowed.  Calls that use the handle's workspace
 *    (xsec_step, me_generate) must not overlap on the device.
 */
#ifndef ME_H_
#define ME_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct me_handle_s *me_handle;

typedef enum {
  ME_OK = 0,
  ME_ERR_ARG = -1,      /* invalid argument (null pointer, size, unknown option) */
  ME_ERR_PROCESS = -2,  /* process name not compiled into this library */
  ME_ERR_CUDA = -3,     /* a CUDA runtime call failed */
  ME_ERR_OOM = -4,      /* device allocation failed */
  ME_ERR_TIMEOUT = -5,  /* a bounded device loop gave up (phase-space redraws exhausted) */
  ME_ERR_STATE = -6     /* call not valid in the handle's state */
} me_status;

typedef enum {
  ME_FP64 = 0,  /* every amplitude operation in FP64 */
  ME_MIXED = 1  /* FP32 amplitudes; FP64 momenta, invariants and propagator denominators */
} me_precision;

/* Standard Model inputs (GeV).  Electroweak scheme: e = sqrt(4 pi alpha),
 * g = e / s_W, g_Z = e / (s_W c_W), v = 2 mW / g.  Fixed widths in every
 * propagator, including t-channel ones (as the paper's HEGET functions).
 *
 * complex_mass != 0 selects the complex-mass option of Sect. 7.11: every
 * vector-boson mass in the couplings becomes mu_V with mu_V^2 = m_V^2 -
 * i m_V Gamma_V (W W H = g mu_W, Z Z H = g_Z mu_Z, v = 2 mu_W / g in H H H,
 * H H H H and t t H), and the W is tied to the Z by mu_W^2 = c_W^2 mu_Z^2, so
 * mW and wW are ignored and c_W mZ, c_W wZ are used everywhere (propagators,
 * the tt~ generator's W Breit-Wigner).  Propagator denominators are the same in
 * both schemes.  reserved_ must be 0. */
typedef struct {
  double alpha, sw2, mZ, wZ, mW, wW, alpha_s, mt, wt, mH, wH;
  int32_t complex_mass;
  int32_t reserved_;
} me_params;

/* Phase-space generators (Sect. 3 and App. A of the paper give its own
 * parametrisation; these are the generators of the workloads). */
typedef enum {
  ME_PS_TWO_BODY = 0,  /* 2 -> 2 at fixed sqrt_s, cos(theta) and phi uniform (massless) */
  ME_PS_RAMBO = 1,     /* flat n-body (RAMBO) at fixed sqrt_s; mass[] per leg, 0 = massless */
  ME_PS_TTBAR = 2,     /* g g > t t~ > (b e+ ve)(b~ e- ve~): sqrt_s uniform in [sqrt_s_min,
                          sqrt_s_max], Breit-Wigner t, t~, W+, W- (Eq. 16, App. A.2), isotropic
                          two-body decays in every rest frame */
  ME_PS_RAMBO_BW = 3,  /* massless final state at fixed sqrt_s whose legs 2 and 3 come from a
                          resonance (res_mass, res_width): dPhi_n = dPhi_{n-1} ds/(2 pi) dPhi_2
                          (App. A.2), s Breit-Wigner mapped over the Eq. 16 range, RAMBO for the
                          resonance and legs 4.., isotropic decay at rest */
  ME_PS_YPT = 4        /* the paper's parametrisation (Eq. 13, App. A.1) at fixed sqrt_s, in the
                          centre-of-mass frame: objects (one leg, or a Breit-Wigner resonance that
                          decays isotropically into two massless legs, App. A.2) in generation order;
                          the first n-2 take y uniform in [-obj_y_max, obj_y_max], the first n-1 take
                          ln(pT^2 + m^2) uniform over [obj_pt_min, obj_pt_max] (Eq. 17; m^2 = s of a
                          resonance) and phi uniform, the last one's pT balances the others, and the
                          longitudinal momentum balance fixes the last two rapidities (two solutions,
                          one drawn).  Their y ranges and the last pT range are checked afterwards.
                          Uniforms: 3 per final leg - 3.  FP64 on both paths. */
} me_ps_kind;

typedef struct {
  int32_t kind;            /* me_ps_kind */
  int32_t max_attempts;    /* redraw limit per point (<= 0: 10000) */
  double sqrt_s;           /* partonic energy (two-body, RAMBO) */
  double sqrt_s_min, sqrt_s_max;  /* range of sqrt(s-hat) (ttbar) */
  double mass[16];         /* on-shell mass per leg (RAMBO); ignored otherwise */
  int32_t n_cut_legs;      /* legs the cuts apply to (0 = no cuts), at most 8 */
  int32_t cut_legs[8];
  double pt_min;           /* pT > pt_min */
  double eta_max;          /* |eta| < eta_max (pseudorapidity) */
  double dr_min;           /* Delta R > dr_min for every pair of cut legs */
  double s_ident;          /* identical-particle factor 1/k! applied to the weights */
  double res_mass, res_width;  /* resonance of ME_PS_RAMBO_BW (GeV) */
  /* ME_PS_YPT objects */
  int32_t n_obj;           /* 2..8; together the objects hold every final leg once */
  int32_t cut_mode;        /* 0: the cuts above (pt_min, eta_max, dr_min on cut_legs); 1: the paper's
                              selection (Eqs. 8-11) by leg_class, with the thresholds below (with
                              ME_PS_YPT only) */
  int32_t obj_legs[8][2];  /* legs of each object (>= 2); obj_legs[j][1] = -1 for a one-leg object */
  int32_t leg_class[16];   /* cut_mode 1: 0 none, 1 jet (|eta| < jet_eta, pT > jet_pt, and
                              min(pT_i, pT_j) Delta R_ij > jet_ptij for every jet pair), 2 b jet,
                              3 charged lepton (pT and |eta| only) */
  double obj_mass[8];      /* mass of a one-leg object */
  double obj_res_mass[8], obj_res_width[8];  /* a two-leg object: its resonance */
  double obj_y_max[8], obj_pt_min[8], obj_pt_max[8];
  double jet_pt, jet_eta, jet_ptij, b_pt, b_eta, lep_pt, lep_eta;  /* cut_mode 1 thresholds */
} me_kin;

/* Monte Carlo accumulator (host).  xsec_step adds to it. */
typedef struct {
  double sum_w;   /* sum of weights, pb */
  double sum_w2;  /* sum of squared weights, pb^2 */
  int64_t n_acc;  /* accepted points */
  int64_t n_try;  /* draws, accepted or not */
} me_xsec_acc;

typedef struct {
  int32_t n_ext;           /* external legs */
  int32_t n_hel;           /* helicity combinations */
  int32_t n_hel_live;      /* combinations evaluated (structural zeros removed) */
  int32_t n_colour;        /* colour basis size K */
  int32_t n_diagrams;      /* Feynman-diagram amplitudes (a 4-gluon vertex counts 3) */
  int32_t pdg[16];         /* PDG code per leg */
  double flops_amp;        /* mixed path: FP32 CUDA-core flops per event (compiler count) */
  double flops_fp64;       /* FP64 path: flops per event (compiler count, colour sum included) */
  double flops_colour;     /* mixed path: colour quadratic-form flops per event run on the tensor
                              cores (algorithmic, 8 K^2 per helicity of the non-root legs);
                              0 where the colour sum is part of flops_amp */
} me_info_t;

/* Create a handle for a compiled process, e.g. "u d~ > e+ ve g g".
 * params: host pointer, NULL for the defaults (alpha = 1/128, sw2 = 0.2312,
 * mZ = 91.1876, wZ = 2.4952, mW = 80.4, wW = 2.085, alpha_s = 0.118,
 * mt = 175, wt = 1.5, mH = 125, wH = 0).  prec: me_precision.
 * Uploads nothing large; allocates no workspace until first needed.
 * Errors: ME_ERR_PROCESS for a name not compiled in, ME_ERR_ARG otherwise. */
me_status me_create(const char *process, const me_params *params, int32_t prec, me_handle *out);

/* |M|^2 (Eq. 4 without the flux and phase space) for n points.
 * momenta: device, n_ext * 4 * n doubles, layout above.  out: device, n
 * doubles.  Asynchronous on stream; n = 0 is a no-op. */
me_status me_eval(me_handle h, const double *momenta, int64_t n, double *out, void *stream);

/* me_eval for host buffers: momenta (n_ext * 4 * n doubles, layout above) and
 * out (n doubles) in host memory, caller-owned.  Page-locked memory that the
 * device maps (cudaHostAlloc / cudaMallocHost, or registered) is read and
 * written by the kernel directly over the CPU-GPU link; other host memory goes
 * through two device buffers in chunks of 2^17 points, copies overlapping the
 * evaluation (buffers kept by the handle until me_destroy).  Synchronous:
 * returns once out holds |M|^2.  Runs on stream (and, for staged memory, a
 * second stream of the handle that follows it).  Errors: ME_ERR_ARG for n < 0,
 * a null pointer or a device pointer; ME_ERR_CUDA. */
me_status me_eval_host(me_handle h, const double *momenta, int64_t n, double *out, void *stream);

/* Phase-space points only: for events counter_offset .. counter_offset+n-1,
 * draw with Philox4x64-10 (counter = (event, attempt, block, 0), key =
 * (seed, 0); each 64-bit word gives two uniforms (w + 1/2) 2^-32 of its 32-bit
 * halves, low half first: uniform i of a draw is half i % 2 of word
 * (i % 8) / 2 of block i / 8) until the cuts pass.  Outputs (device, any may be NULL):
 * momenta (n_ext * 4 * n, layout above), weight (n: phase-space weight),
 * shat (n), tries (n: draws used).  Asynchronous on stream.  A point that
 * exhausts kin->max_attempts is reported by the next synchronising call on
 * the handle as ME_ERR_TIMEOUT. */
me_status me_generate(me_handle h, uint64_t seed, uint64_t counter_offset, int64_t n, const me_kin *kin,
                      double *momenta, double *weight, double *shat, int32_t *tries, void *stream);

/* One Monte Carlo step over n_accept accepted points (events
 * counter_offset .. counter_offset+n_accept-1): generate, cut, evaluate,
 * weight w = W_PS |M|^2 s_ident / (2 s-hat) * 0.3893793721e9 pb GeV^2, and add
 * (sum w, sum w^2, n_acc, n_try) to *acc (host).  The sums are reduced
 * deterministically.  Optional device outputs (NULL to skip): me2_out (n_accept
 * doubles), momenta_out (layout above).  Synchronises stream before
 * returning.  Errors: ME_ERR_TIMEOUT if a point exhausted its redraws. */
me_status xsec_step(me_handle h, uint64_t seed, uint64_t counter_offset, int64_t n_accept, const me_kin *kin,
                    void *stream, me_xsec_acc *acc, double *me2_out, double *momenta_out);

/* xsec_step without a host synchronisation, for back-to-back steps: the
 * step's sums are added on the device, after its kernels and in the same fixed
 * order as xsec_step, to acc_dev[0..3] = (sum of weights in pb, sum of squared
 * weights, draws, number of steps in which a point exhausted its redraws).
 * acc_dev: device memory, 4 doubles, caller-owned and initialised (zeros for a
 * new estimate); n_acc is the sum of the steps' n_accept.  Returns once the
 * work is queued on stream; argument errors return synchronously, a device
 * error at the next synchronising call.  Steps on one handle share its
 * workspace and must be queued on one stream (or otherwise ordered).  The
 * per-kernel timing of me_step_timing does not apply. */
me_status xsec_step_async(me_handle h, uint64_t seed, uint64_t counter_offset, int64_t n_accept,
                          const me_kin *kin, void *stream, double *acc_dev);

/* xsec_step for callers that cannot allocate device memory: the same
 * computation and arguments, but the step's scratch (per-block partial sums,
 * totals, status flag) lives in a fixed array compiled into the library
 * instead of memory the library would cudaMalloc.  Such callers include code
 * running inside a host application that owns all device memory through its
 * own pool or arena, or that forbids allocations after start-up; cudaMalloc
 * there either fails or breaks the owner's accounting.  This entry point calls
 * no cudaMalloc, cudaFree or allocating library routine.  (It has no
 * counterpart in the paper; it exists for embedding.)
 *  - Limit: the fused kernel's grid (at most 8 blocks per SM) must fit the
 *    scratch's 4096 partial slots; larger launches are rejected with
 *    ME_ERR_ARG.  The array occupies about 100 KB on every GPU that loads the
 *    library, until the process exits.
 *  - The first call on a device looks up the array's device address (with that
 *    device current), and so does the first call after the device's context
 *    was made anew (cudaDeviceReset); make those calls before any stream
 *    capture.
 *  - Processes whose |M|^2 kernel takes one event per block (the all-gluon
 *    processes) have no fused step: ME_ERR_ARG, before any device work.
 *  - Every call shares the one array: calls whose work overlaps on the GPU (on
 *    different streams, or from several threads) race and corrupt each other's
 *    sums.  Serialise them.  The array keeps the previous call's contents; the
 *    call clears the status flag itself and overwrites the rest.
 *  - me2_out, momenta_out: optional device outputs as in xsec_step.
 * Synchronises stream before returning. */
me_status xsec_step_noalloc(me_handle h, uint64_t seed, uint64_t counter_offset, int64_t n_accept,
                            const me_kin *kin, void *stream, me_xsec_acc *acc, double *me2_out,
                            double *momenta_out);

/* Per-kernel device time of xsec_step, from CUDA events recorded on the call's
 * stream around the phase-space kernel and the amplitude kernel of every chunk.
 * Writes the sums (ms) accumulated since the previous call to *ms_ps and
 * *ms_me (either may be NULL), resets them, and turns recording on (enable = 1)
 * or off (0).  While on, xsec_step waits for each chunk's events.  (No
 * counterpart in the paper; a measurement aid.) */
me_status me_step_timing(me_handle h, int32_t enable, double *ms_ps, double *ms_me);

/* ---------------------------------------------------------------------------
 * Adaptive integration: VEGAS grids (G. P. Lepage, J. Comput. Phys. 27 (1978)
 * 192), the role of the BASES / gBASES integrator the paper uses for its cross
 * sections (Sect. 6).  A grid holds, for each uniform variable the phase-space
 * generator draws (2 for the two-body generator, 4 per final-state particle for
 * RAMBO, 15 for the tt~ chain), n_bins bin edges 0 = e_0 < ... < e_N = 1,
 * stored [dimension][N + 1].  A uniform y in bin i = floor(N y) maps to
 * e_i + (N y - i)(e_{i+1} - e_i) and the weight is multiplied by the map's
 * Jacobian prod_d N (e_{d,i+1} - e_{d,i}).  Host-side object; device buffers
 * are owned by the grid.
 * ------------------------------------------------------------------------- */
typedef struct me_grid_s *me_grid;

/* Equal bins for the generator and cuts of kin on handle h's process.
 * n_bins: 1..256, with dimensions * n_bins <= 6144. */
me_status me_grid_create(me_handle h, const me_kin *kin, int32_t n_bins, me_grid *out);
me_status me_grid_info(me_grid g, int32_t *n_dims, int32_t *n_bins);
/* Host copies of the edges, [n_dims][n_bins + 1]; set checks 0 .. 1 and increase. */
me_status me_grid_get_edges(me_grid g, double *edges);
me_status me_grid_set_edges(me_grid g, const double *edges);
/* Histogram of the refinement, [n_dims][n_bins]: sum of w^2 over the accepted
 * points of the grid steps since the last refine or clear whose uniform of that
 * dimension fell in that bin.  Summed with atomics: equal to rounding, not
 * bitwise, between runs. */
me_status me_grid_get_hist(me_grid g, double *hist);
me_status me_grid_clear_hist(me_grid g);
/* New edges from the histogram (per dimension: neighbour smoothing of the bin
 * sums, normalisation r_i, damping ((1 - r_i) / ln(1 / r_i))^alpha, equal shares
 * of the damped weights per new bin; a dimension with no weight keeps its
 * edges), then clears the histogram.  alpha > 0 (1.5 is customary). */
me_status me_grid_refine(me_grid g, double alpha);
/* The same refinement on host arrays, no device involved: edges and out
 * [n_dims][n_bins + 1], hist [n_dims][n_bins]. */
me_status me_vegas_refine_edges(const double *edges, const double *hist, int32_t n_dims, int32_t n_bins, double alpha,
                                double *out);
/* xsec_step with every uniform mapped through the grid and the weights
 * carrying its Jacobian; adds the points' squared weights to the grid's
 * histogram.  The grid must come from the same process and generator kind.
 * One step at a time per grid (its per-chunk buffers are shared). */
me_status xsec_step_grid(me_handle h, me_grid g, uint64_t seed, uint64_t counter_offset, int64_t n_accept,
                         const me_kin *kin, void *stream, me_xsec_acc *acc, double *me2_out, double *momenta_out);
void me_grid_destroy(me_grid g);

/* sigma-hat = sum_w / n_try and its standard error (pb) from an accumulator. */
me_status me_xsec_estimate(const me_xsec_acc *acc, double *sigma, double *error);

me_status me_info(me_handle h, me_info_t *info);

/* Number of processes compiled into the library and their names. */
int32_t me_n_processes(void);
const char *me_process_name(int32_t i);

void me_destroy(me_handle h);
const char *me_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ME_H_ */

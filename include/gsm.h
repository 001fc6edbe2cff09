/*
 * gsm.h - C ABI of the B300 (sm_103a) Generalized Source Method solver for 3D
 * periodic dielectric composites (Shcherbakov & Tishchenko, arXiv:1501.01752).
 *
 * The library solves the truncated Fourier-space equation of the paper's GSM
 * section (Eq. 4),
 *
 *   E_{a m} = E^inc_{a m} + sum_b G_ab(m) sum_{m'} (Delta eps/eps_b)_{m-m'} E_{b m'},
 *   G_ab(m) = (k_b^2 delta_ab - k_{a m} k_{b m}) / (k_m^2 - k_b^2),
 *   k_{a m} = k^inc_a + m_a K_a,  K_a = 2 pi / Lambda_a,  k_b^2 = k0^2 eps_b,
 *   E^inc_{a m} = delta_{m 0} a_a,
 *
 * with a Krylov method whose matrix-vector product is a pruned 3D FFT
 * convolution (the Toeplitz product) followed by the per-harmonic Green tensor.
 * It sweeps |k_inc| = kappa, fits the resonance poles of the 0th-order
 * response (Eqs. 6-10 of the "Modes in 3D crystals" section) and returns the
 * principal effective permittivities eps_aa = (eta / k0)^2.  An adjoint solve
 * gives gradients with respect to voxel permittivities.
 *
 * Conventions used by every call:
 *   - Units: lengths in vacuum wavelengths is the usual choice (k0 = 2 pi);
 *     any consistent unit works since only k0 * Lambda enters.
 *   - Field layout: per instance 3 planar components, each N_z x N_y x N_x
 *     complex128 (interleaved re, im), x fastest; harmonic m sits at index
 *     (m_z + n_z, m_y + n_y, m_x + n_x) with n_a = (N_a - 1) / 2.
 *   - Fourier convention: eps(r) = sum_m eps_m exp(i K_m . r); a shape
 *     centred at c contributes (eps_s - eps_host) exp(-i K_m . c) chi_s(K_m).
 *   - Ownership: the plan owns all device memory it allocates; arrays passed
 *     by the caller stay the caller's and are not retained after return.
 *   - Streams: work is issued on desc.cuda_stream (0 = legacy default) and
 *     every call synchronises that stream before it returns.
 *   - Errors: every call returns a gsm_status; nothing is thrown across the
 *     ABI.  gsm_last_error(plan) gives a one-line message.  On an error other
 *     than GSM_ERR_NOCONV, output arrays are left untouched.
 *   - Threads: a plan may be used by one host thread at a time.
 */
#ifndef GSM_H
#define GSM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GSM_OK = 0,
  GSM_ERR_ARG = 1,      /* invalid argument (message names it)                 */
  GSM_ERR_SINGULAR = 2, /* some harmonic has k_m^2 ~= k_b^2 (Eq. 4 undefined)  */
  GSM_ERR_NOCONV = 3,   /* Krylov solve missed tol within max_iter; best iterate written */
  GSM_ERR_NOMEM = 4,    /* device allocation failed or hbm cap too small       */
  GSM_ERR_CUDA = 5,     /* CUDA runtime error (message has the CUDA string)    */
  GSM_ERR_TIMEOUT = 6,  /* reserved for bounded device waits                   */
  GSM_ERR_STATE = 7     /* call out of order (e.g. solve before permittivity)  */
} gsm_status;

enum { GSM_FP64 = 0, GSM_FP32_REFINE = 1 };          /* arithmetic of the solve  */
/* gsm_apply only: the FP64-accurate product computed in double-float
 * arithmetic (each real an unevaluated sum of two FP32 values, ~48
 * significand bits), the arithmetic of the outer residual of refined solves */
enum { GSM_DF64 = 2 };
/* outer residual b - A x of GSM_FP32_REFINE solves: double-float on the
 * FP32 pipes where the lane-team product applies (FFT sizes 32/64), FP64
 * otherwise (AUTO), or FP64 always */
enum { GSM_RESID_AUTO = 0, GSM_RESID_FP64 = 1 };
/* the field the plan solves for: E of Eq. 4, or H of Eq. 5 (the H-field
 * formulation, with the Fourier coefficients of 1/eps; point pol is then the
 * incident H amplitude and the output field is H) */
enum { GSM_FORM_E = 0, GSM_FORM_H = 1 };
enum { GSM_GMRES = 0, GSM_BICGSTAB = 1 };            /* Krylov method            */
/* Krylov solves of Eq. 4 with the lane-team product (FFT sizes 32/64, cubic
 * 128) and a contrast |Delta_0| = |<eps>/eps_b - 1| >= 1: right
 * preconditioner M = I - s Delta_0 G(m), the block diagonal of Eq. 4 (the
 * Green tensor of the cell-averaged medium, inverted in closed form per
 * harmonic; s in {1, 1/2, 1/4, 1/8} per point keeps M away from singular,
 * s = 0 when no choice does), or none.  The solution is the same; only the
 * number of Krylov steps changes.  Not in the paper. */
enum { GSM_PRECOND_AUTO = 0, GSM_PRECOND_NONE = 1 };
enum { GSM_SPHERE = 0, GSM_BOX = 1, GSM_ELLIPSOID = 2 };

typedef struct gsm_plan_s gsm_plan_t;

/* Plan description (GSM section: truncation to N_x x N_y x N_z harmonics;
 * "Calculation details": GMRES in Saad's form). */
typedef struct {
  double period[3];     /* Lambda_x, Lambda_y, Lambda_z (> 0)                            */
  int n_harm[3];        /* N_x, N_y, N_z: odd, >= 1, <= 127                              */
  int fft[3];           /* FFT points per axis >= 2N-1: 0 = smallest power of two (<= 256);
                           a power of two or 3 * 2^p in [24, 192] as given; -1 = tuned
                           per level (see gsm_level_fft)                                 */
  double eps_b[2];      /* basis permittivity eps_b (re, im); im must be 0               */
  int precision;        /* GSM_FP64 or GSM_FP32_REFINE                                   */
  int krylov;           /* GSM_GMRES (basis of restart + 1 vectors per instance) or
                           GSM_BICGSTAB (seven vectors per instance, no restart)          */
  int restart;          /* GMRES basis length m; 0 = 60                                  */
  int max_iter;         /* total matrix-vector products per instance; 0 = 2000           */
  double tol;           /* target ||b - A x|| / ||b||; 0 = 1e-8                          */
  double inner_tol;     /* FP32 inner GMRES relative tolerance; 0 = 1e-4                 */
  int max_batch;        /* instances solved together; 0 = 32                             */
  size_t hbm_cap_bytes; /* 0 = unlimited; bounds the Krylov basis (restart shrinks)      */
  int device;           /* CUDA device ordinal                                           */
  void *cuda_stream;    /* cudaStream_t to issue work on; NULL = default stream          */
  int residual;         /* GSM_RESID_AUTO or GSM_RESID_FP64 (refined solves)             */
  int form;             /* GSM_FORM_E (Eq. 4) or GSM_FORM_H (Eq. 5)                      */
  int precond;          /* GSM_PRECOND_AUTO (GMRES on Eq. 4, lane-team levels) or NONE    */
} gsm_plan_desc;

/* Non-overlapping inclusion in the host medium (GSM section: analytic Fourier
 * images of simple shapes, combined).  size: SPHERE radius in size[0]; BOX
 * full side lengths; ELLIPSOID semi-axes.  center in [0, Lambda) per axis. */
typedef struct {
  int kind;
  double center[3];
  double size[3];
  double eps[2];        /* (re, im); im must be 0 */
} gsm_shape;

/* One incident plane wave (text after Eq. 4): |k_inc| = kappa along kdir,
 * polarisation a (complex 3-vector, interleaved), frequency k0 = omega/c. */
typedef struct {
  double k0;
  double kdir[3];       /* need not be normalised                                   */
  double kappa;
  double pol[6];        /* a_x re, a_x im, a_y re, a_y im, a_z re, a_z im            */
  int n_harm[3];        /* 0 = plan's N; otherwise odd and <= plan's N per axis     */
} gsm_point;

typedef struct {
  int iters;            /* matrix-vector products of the Krylov method                */
  int refine_steps;     /* outer FP64 residual evaluations                             */
  double rel_residual;  /* final FP64 ||b - A x|| / ||b||                              */
  int status;           /* gsm_status of this instance                                 */
} gsm_info;

/* Host-only query (no device needed): the FFT sizes the plan would use and
 * its device memory estimate in bytes.  Returns GSM_ERR_ARG on a bad desc. */
gsm_status gsm_plan_query(const gsm_plan_desc *desc, int fft_out[3], size_t *bytes_out);

/* Create a plan on desc->device.  Allocates the FFT twiddle tables and the
 * per-level workspace lazily.  *out is NULL on failure. */
gsm_status gsm_plan(const gsm_plan_desc *desc, gsm_plan_t **out);
void gsm_plan_destroy(gsm_plan_t *plan);

/* Set eps(r) of the unit cell ("Calculation details": analytic Fourier images).
 * Either n_shapes >= 0 inclusions in a host of eps_host, or (voxel_eps != NULL)
 * a grid of M[0] x M[1] x M[2] constant voxels (real eps, x fastest, voxel
 * (vx,vy,vz) fills [v_a, v_a+1) Lambda_a / M_a), whose Fourier coefficients
 * are exact integrals.  Shapes and voxels together are GSM_ERR_ARG; complex
 * eps is GSM_ERR_ARG (lossless media only).  Builds the convolution
 * multiplier D(r) = sum_d (Delta eps/eps_b)_d exp(2 pi i d.r/L) / (L_x L_y L_z)
 * on the device for each truncation used. */
gsm_status gsm_set_permittivity(gsm_plan_t *plan, const double eps_host[2],
                                const gsm_shape *shapes, int n_shapes,
                                const double *voxel_eps, const int M[3]);

/* y = op(A) x for n points, each x/y of 3 N^3 complex128 (point's
 * truncation), A the plan's operator (Eq. 4, or Eq. 5 for a GSM_FORM_H plan):
 *   op = 0: y = A x;
 *   op = 1: y = A^H x (Eq. 4 only);
 *   op = 2: y = A M^{-1} x, the right-preconditioned Eq. 4 operator that the
 *           Krylov solves iterate with (GSM_PRECOND_AUTO above: lane-team
 *           levels with |Delta_0| >= 1 and points that get s > 0, else
 *           GSM_ERR_ARG), run by the same kernels as inside a solve.  Not in
 *           the paper.
 * on_device = 1: x, y are device pointers; 0: host.  precision
 * GSM_FP32_REFINE rounds x to complex64 and applies the FP32 kernels (result
 * widened to complex128); GSM_DF64 applies the double-float kernels (op = 0
 * and FFT sizes 32 or 64 only, else GSM_ERR_ARG). */
gsm_status gsm_apply(gsm_plan_t *plan, int n, const gsm_point *points,
                     const double *x, double *y, int on_device, int precision, int op);

/* Solve Eq. 4 for n points (any n; processed in batches of max_batch).  E
 * receives n fields of 3 N^3 complex128 (on_device selects device or host
 * memory).  infos (n entries) may be NULL.  Returns GSM_ERR_NOCONV if any
 * instance missed tol (its best iterate is written), GSM_ERR_SINGULAR if a
 * harmonic of some point lies on the basis light cone. */
gsm_status gsm_solve(gsm_plan_t *plan, int n, const gsm_point *points,
                     double *E, int on_device, gsm_info *infos);

/* As gsm_solve but returns only the 0th harmonic E_0 (3 complex128 per point,
 * host memory): the response of the "Modes in 3D crystals" section. */
gsm_status gsm_sweep(gsm_plan_t *plan, int n, const gsm_point *points,
                     double *E0, gsm_info *infos);

/* Pole fit of Eqs. 7-10 (host, FP64): kappa[n] equidistant real, xi[n]
 * complex (interleaved).  Needs Nd > Np and n >= Nd + Np.  eta, zeta receive
 * Np complex values each. */
gsm_status gsm_fit_poles(int n, const double *kappa, const double *xi, int Np, int Nd,
                         double *eta, double *zeta);

/* Principal effective permittivities (numerical-convergence section:
 * principal axes along x, y, z): three sweeps of n_kappa equidistant points
 * over kappa_lo_hi[c][0..1] with (kdir, a) = (z, x), (z, y), (x, z); fit; the
 * largest-residue pole inside each interval gives eps_cc = (eta/k0)^2.
 * diag (may be NULL) receives per component: eta (2), zeta (2). */
gsm_status gsm_retrieve_tensor(gsm_plan_t *plan, double k0, const double kappa_lo_hi[6],
                               int n_kappa, int Np, int Nd, double eps_eff[3], double *diag);

/* Adjoint gradient (no counterpart in the paper; the calculus of Eq. 4): for
 * n points with objective gradients gE0 (3 complex per point, dL/dRe E_0 +
 * i dL/dIm E_0), accumulate dL/d eps_v into grad_voxel (host, M[0]M[1]M[2]
 * reals, x fastest) for the voxel structure last set.  Requires a voxel
 * permittivity.  Solves A E = b and A^H lambda = g~ per point. */
gsm_status gsm_adjoint(gsm_plan_t *plan, int n, const gsm_point *points,
                       const double *gE0, double *grad_voxel);

/* Gradient of sum_c weights[c] Re eps_cc (the retrieval above) with respect
 * to every voxel permittivity: sweeps, pole fits, pole sensitivities and
 * adjoint solves.  eps_eff receives the retrieved diagonal. */
gsm_status gsm_retrieve_tensor_grad(gsm_plan_t *plan, double k0, const double kappa_lo_hi[6],
                                    int n_kappa, int Np, int Nd, const double weights[3],
                                    double eps_eff[3], double *grad_voxel);

/* Per-kernel timing with CUDA events on the plan's stream.  enable = 1 starts
 * recording (and clears totals); gsm_profile_get returns launches, summed
 * device milliseconds and algorithmic bytes for kernel class `kind`
 * (0 x-forward, 1 yz-convolution, 2 x-inverse+Green (these three: the
 * working-precision product), 3 Krylov dots, 4 Krylov update, 5 other,
 * 6 FP64 residual product (all three passes); 7 = number of kernels the
 * plan launched since gsm_profile, counted whether or not recording is on). */
gsm_status gsm_profile(gsm_plan_t *plan, int enable);
gsm_status gsm_profile_get(gsm_plan_t *plan, int kind, long long *launches,
                           double *total_ms, double *bytes);

/* y = A x for ONE point at the plan's full truncation, with the plan's
 * operator (Eq. 4, or Eq. 5 for a GSM_FORM_H plan) in FP64 kernels, without
 * allocating anything.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc during a
 * solve step -- host applications whose own allocator has reserved the
 * device memory up front, or latency-critical loops in which the implicit
 * synchronisation of an allocation is not acceptable.  x and y are device
 * pointers to 3 N^3 complex128 (y must not alias x).  Every temporary lives
 * in one fixed device array of 8 MiB that the library holds on each GPU
 * until the process exits; truncations whose temporaries (3 L_x N_y N_z
 * complex128 plus 12 N^3 bytes) exceed it return GSM_ERR_ARG.  The first
 * call on a device looks up that array's device address (once per device),
 * so make the first call before any stream capture.  All calls share the
 * array: calls that overlap on the GPU (other streams, other plans) race and
 * must be serialised by the caller.  The plan must have its permittivity
 * set; the call synchronises the plan's stream. */
gsm_status gsm_apply_noalloc(gsm_plan_t *plan, const gsm_point *point, const double *x, double *y);

/* Threads per block that the autotuner chose for the three passes of the
 * lane-team product (FFT sizes 32/64) of the plan's full truncation in the
 * given precision: each pass is timed at 128, 256 and 512 threads on the
 * first batch solved and the fastest is kept (256 before that, or with
 * GSM_AUTOTUNE=0 in the environment).  GSM_ERR_STATE before the first solve. */
gsm_status gsm_tuned_blocks(const gsm_plan_t *plan, int precision, int blocks[3]);

/* FFT grid (points per axis) of the level of truncation n_harm once it has
 * been built by a call on points of that truncation: the plan's sizes, or,
 * for axes given as fft = -1, the power of two or the smaller mixed-radix
 * size 3 * 2^p, whichever ran one product of the batch faster when the level
 * was first built.  GSM_ERR_STATE if the level does not exist yet. */
gsm_status gsm_level_fft(const gsm_plan_t *plan, const int n_harm[3], int fft_out[3]);

/* Measured fused multiply-add throughput of `device` (no counterpart in the
 * paper): the denominator of the arithmetic rooflines (FP64 product,
 * double-float residual).  kind 0: FP64 FMA, 1: FP32 FMA, 2: packed FP32
 * pairs (fma.rn.f32x2).  One wave of 256-thread blocks per SM slot, eight
 * independent chains per thread, best of five launches timed with CUDA
 * events on cuda_stream (NULL = default stream); *tflops = 2 x FMAs / s.
 * Allocates and frees a small result buffer; changes no device setting.
 * GSM_ERR_ARG for a null tflops or another kind, GSM_ERR_CUDA if the device
 * cannot be selected or a launch fails, GSM_ERR_NOMEM if the buffer cannot
 * be allocated. */
gsm_status gsm_probe_fma(int device, void *cuda_stream, int kind, double *tflops);

const char *gsm_last_error(const gsm_plan_t *plan);
const char *gsm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GSM_H */

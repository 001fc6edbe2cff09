// Host-side declarations of the kernel launchers and the per-kernel event
// profiler shared by the CUDA translation units.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "dfloat.cuh"

namespace gsm {

constexpr int TWN_HOST = 768;  // twiddle table entries: exp(2 pi i j / 768), every supported FFT size divides 768

enum ProfKind { KIND_FWD_X = 0, KIND_YZ = 1, KIND_INV_X = 2, KIND_DOTS = 3, KIND_UPDATE = 4, KIND_OTHER = 5,
                KIND_RESID64 = 6, KIND_COUNT = 7 };

// Records a CUDA event pair around each launch of a kernel class on the
// launching stream; durations are summed when read.
struct Profiler {
  bool on = false;
  struct Rec { cudaEvent_t a, b; int kind; double bytes; };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  cudaEvent_t pending_begin = nullptr;
  long long launches[KIND_COUNT] = {0};
  double ms[KIND_COUNT] = {0};
  double bytes[KIND_COUNT] = {0};

  cudaEvent_t get() {
    if (used < pool.size()) return pool[used++];
    cudaEvent_t e;
    cudaEventCreate(&e);
    pool.push_back(e);
    used++;
    return e;
  }
  void begin(int, cudaStream_t st) {
    pending_begin = get();
    cudaEventRecord(pending_begin, st);
  }
  void end(int kind, cudaStream_t st, double nbytes) {
    cudaEvent_t e = get();
    cudaEventRecord(e, st);
    recs.push_back({pending_begin, e, kind, nbytes});
  }
  // fold recorded pairs into totals (stream must be synchronised)
  void collect() {
    for (auto &r : recs) {
      float t = 0;
      cudaEventElapsedTime(&t, r.a, r.b);
      launches[r.kind] += 1;
      ms[r.kind] += t;
      bytes[r.kind] += r.bytes;
    }
    recs.clear();
    used = 0;
  }
  void reset() {
    recs.clear();
    used = 0;
    for (int k = 0; k < KIND_COUNT; ++k) { launches[k] = 0; ms[k] = 0; bytes[k] = 0; }
  }
  ~Profiler() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

template <typename R> struct MatvecArgs {
  using C = typename Cx<R>::T;
  using IO = typename Io<R>::T;
  Geo g;
  int B = 0;
  IO *X = nullptr;         // input field(s), instance stride xstride
  long long xstride = 0;
  IO *Y = nullptr;         // output field(s), instance stride ystride (never aliases X)
  long long ystride = 0;
  C *T = nullptr;          // intermediate, B * g.Tsz complex
  const R *D = nullptr;    // convolution multiplier [rx][ry][rz]
  const float2 *Dp = nullptr;  // complex64 only: D as x-plane pairs [rx / 2][ry][rz] (nullptr = unpaired pass 2)
  const R *scale = nullptr;  // per-instance input scale (nullptr = 1)
  const int *act = nullptr;
  const Inst *inst = nullptr;
  const R *iden = nullptr; // [B][Nh] 1/(k_m^2 - k_b^2)
  const C *tw = nullptr;   // 256-entry twiddle table
  int mode = 0;            // 0: A x, 1: b - A x, 2: A^H x, 3: b - A^H x
  int form = 0;            // 0: Eq. 4 (E field), 1: Eq. 5 (H field; modes 0 and 1 only)
  int pc = 0;              // 1: Y = A M^{-1} X with the right preconditioner of Inst (Eq. 4, mode 0,
                           // lane-team path only)
  double *partial = nullptr;
  unsigned *counter = nullptr;
  double *norm_out = nullptr;  // ||Y||^2 per instance (nullptr = skip)
  const int *jdev = nullptr;   // graph mode: X and Y advance by (*jdev) * jstride
  long long jstride = 0;
  int nact = 0;                // profiling only: instances still active (0 = all B), for the byte count
  int yzv = 1;                 // complex64 pass 2: 1 = lane-shuffle transposes (k_yz_t8x2r),
                               // 0 = team-buffer transposes (k_yz_t8x2)
};

template <typename R> cudaError_t launch_matvec(const MatvecArgs<R> &a, cudaStream_t st, Profiler *prof);
// team-of-lanes FFT path for FFT sizes 32/64 on every axis, cubic 128 (modes
// 0, 1; modes 2, 3 for Eq. 4)
bool reg_path_ok(const Geo &g);
template <typename R>
cudaError_t launch_matvec_reg(const MatvecArgs<R> &a, cudaStream_t st, Profiler *prof, const int *tb);
// one pass (1, 2, 3) with block size tb in {128, 256, 512} (autotuner)
template <typename R> cudaError_t launch_reg_pass(int pass, int tb, const MatvecArgs<R> &a, cudaStream_t st);
// x-plane pairs of the complex64 multiplier for the packed pass 2
cudaError_t launch_pair_d(const float *D, float2 *Dp, const Geo &g, cudaStream_t st);
bool packed_yz_ok(const Geo &g);
int matvec_reg_blocks_pass3(const Geo &g);
int matvec_blocks_pass3(const Geo &g, size_t csize);
size_t matvec_max_smem(const Geo &g, size_t csize);
cudaError_t launch_iden(const Geo &g, const Inst *inst, int B, double *id64, float *id32, cudaStream_t st,
                        dfl *iddf = nullptr);
cudaError_t launch_d2df(const double *in, dfl *out, long long n, cudaStream_t st);
cudaError_t launch_convert_d2f(const double2 *in, float2 *out, long long n, cudaStream_t st);
cudaError_t launch_convert_f2d(const float2 *in, double2 *out, long long n, cudaStream_t st);

// generic FP64 FFT along one axis of a batch of [Lz][Ly][Lx] complex arrays
cudaError_t launch_fft_axis(double2 *data, int Lx, int Ly, int Lz, int axis, int sign, int batch,
                            long long batch_stride, const double2 *tw, cudaStream_t st);
cudaError_t launch_d_finalize(const double2 *Dc, const Geo &g, double scale, double *D64, float *D32,
                              cudaStream_t st);

// Krylov kernels (krylov.cu)
struct KrylovPtrs {
  int B, m;
  long long U;              // logical vector length (3 N^3)
  long long Us;             // stored stride: U rounded up to 64 (pads stay zero)
  int nblk;                 // blocks per instance for vector kernels
  int bcap;                 // most blocks per instance, one per 2048 elements: the Gram-Schmidt
                            // passes spread nblk * B blocks over the active instances.  2048 is the
                            // FP32 update's tile; k_dots tiles hold 1024 (FP32) or 512 (FP64)
                            // elements and the FP64 update's 1024, so there a lone instance gets
                            // fewer blocks than tiles and each block loops over several tiles
  int *alist;               // [B + 1]: number of active instances, then their indices
  double *partial;          // [B][nblk][2(m+1)+1]
  unsigned *counter;        // [B]
  double *hdot0, *hdot1;    // [B][2(m+1)+1] dots (+ ||w||^2 last)
  double *wn0, *wn1;        // [B] ||w||^2 after update passes
  int *gate;                // [B] reorthogonalise flag
  int *act;                 // [B] Arnoldi active
  double2 *H;               // [B][m][m+1] rotated Hessenberg columns
  double *cs;               // [B][m]
  double2 *sn;              // [B][m]
  double2 *gv;              // [B][m+1]
  double2 *y;               // [B][m]
  double *thresh;           // [B]
  int *kcount;              // [B]
  float *scale32;           // [B] 1 / ||v_j|| of the vector the next product takes
  double *scale64;          // [B]
  double *dnorm2;           // [B] ||d||^2 of the correction added to x by the last solution update
  double *dpartial;         // [B][nblk] its block partials (shared with the product's norm partials)
  unsigned *dcounter;       // [B] its last-block counters
  long long *ulen;          // [B] stored length of each instance's vectors (U_b rounded up to 64), for
                            // batches of several truncations; the vector stride stays Us.
                            // Uniform batches pass nullptr to the kernels (every length Us)
  double *svec;             // [B][m+1] 1 / ||v_i|| of every stored basis vector: GMRES keeps the
                            // basis unnormalised (v_i = svec_i * V_i), the scales enter the dots,
                            // the update coefficients and the solution update
  double *resid;            // [B]
  int force_reorth;         // 0: DGKS test, 1: always reorthogonalise, 2: never, k >= 3: every 2^(k - 2)-th step
  int nact;                 // profiling only: instances active in the step launched (0 = all B);
                            // the recorded bytes of the Gram-Schmidt passes count these
  int *jdev;                // graph mode: Arnoldi step counter on the device (nullptr: host j)
};

template <typename R>
cudaError_t launch_arnoldi_ortho(const KrylovPtrs &k, typename Cx<R>::T *V, long long vinst, int j, cudaStream_t st,
                                 Profiler *prof);
cudaError_t launch_finish(const KrylovPtrs &k, int j, cudaStream_t st);
// graph mode: j += 1 and set the WHILE condition (any instance active and j < m)
cudaError_t launch_advance(const KrylovPtrs &k, cudaGraphConditionalHandle h, cudaStream_t st);
cudaError_t launch_backsolve(const KrylovPtrs &k, cudaStream_t st);
template <typename R>
cudaError_t launch_sol_update(const KrylovPtrs &k, double2 *x64, long long xinst, typename Cx<R>::T *V,
                              long long vinst, const int *need, int dslot, cudaStream_t st, Profiler *prof);
// right-preconditioned cycles: u = V y (GMRES, src < 0) or u = V[src]
// (BiCGSTAB), x += M^{-1} u per harmonic (M^{-1} of Inst with the product's
// 1/(k_m^2 - k_b^2) in the basis precision); u kept in slot dslot if >= 0
template <typename R>
cudaError_t launch_sol_update_pc(const KrylovPtrs &k, const Geo &g, const Inst *inst, const R *iden, double2 *x64,
                                 long long xinst, typename Cx<R>::T *V, long long vinst, const int *need, int dslot,
                                 int src, cudaStream_t st, Profiler *prof);
cudaError_t launch_resid_sub(double2 *r64, long long rinst, const float2 *Ad, long long ainst, long long U, int B,
                             int nblk, const int *need, double *partial, unsigned *counter, double *norm_out,
                             cudaStream_t st);
template <typename C>
cudaError_t launch_start_basis(const double2 *r64, long long rinst, C *V, long long vinst, long long U, int B,
                               int nblk, const int *need, cudaStream_t st);
template <typename C>
cudaError_t launch_zero_pads(C *V, long long nvec, long long U, long long Us, cudaStream_t st);
cudaError_t launch_set_rhs(double2 *r64, long long xinst, const Geo &g, const Inst *inst, int B, cudaStream_t st);
cudaError_t launch_extract_e0(const double2 *x64, long long xinst, const Geo &g, int B, double2 *out,
                              cudaStream_t st);

// BiCGSTAB (bicgstab.cu): seven vectors per instance in the working
// precision, scalars in FP64.  Slots of V[b][slot][Us]:
enum { BS_R = 0, BS_RH = 1, BS_P = 2, BS_V = 3, BS_S = 4, BS_T = 5, BS_D = 6, BS_COUNT = 7 };
// kernels of one iteration, in order (BICG_INIT once per cycle)
enum { BICG_INIT = 0, BICG_P = 1, BICG_ALPHA = 2, BICG_S = 3, BICG_OMEGA = 4, BICG_UPDATE = 5 };
struct BicgPtrs {
  int B;
  long long U, Us;          // logical and stored vector length
  int nblk;                 // blocks per instance
  double *partial;          // [B][nblk][3] block partial sums
  unsigned *counter;        // [B] last-block counters (zero between kernels)
  double2 *sc;              // [B][4] rho, rho_old, alpha, omega
  double *rn2;              // [B] ||r||^2 of the inner residual
  double *thresh2;          // [B] stop when ||r||^2 <= thresh2
  int *act;                 // [B] instance still iterating
  int *it;                  // [B] iterations of this cycle
  int max_it;               // iteration cap of a cycle
  double *dnorm2;           // [B] ||d||^2 of the correction added to x (k_bicg_sol)
  double *dpartial;         // [B][nblk] its block partials
  unsigned *dcounter;       // [B] its last-block counters
};
template <typename R>
cudaError_t launch_bicg_step(int which, const BicgPtrs &bp, typename Cx<R>::T *V, long long vinst, cudaStream_t st);
template <typename R>
cudaError_t launch_bicg_sol(double2 *x64, long long xinst, const typename Cx<R>::T *V, long long vinst,
                            const BicgPtrs &bp, const int *need, cudaStream_t st);
cudaError_t launch_bicg_advance(const BicgPtrs &bp, cudaGraphConditionalHandle h, cudaStream_t st);

// adjoint gradient (adjoint.cu)
cudaError_t launch_adj_scatter(const Geo &g, const double2 *lam, const double2 *E, const Inst *inst, const double *iden,
                               double2 *grid, cudaStream_t st);
cudaError_t launch_adj_accum(const double2 *grid, long long LL, double2 *P, cudaStream_t st);
cudaError_t launch_adj_fold(const double2 *P, const Geo &g, const int M[3], double2 *Q, cudaStream_t st);
cudaError_t launch_adj_real(const double2 *Q, long long n, double scale, double *out, cudaStream_t st);

// read-only view of a plan for entry points outside api.cu
struct PlanView {
  Geo g;
  int form;                // 0: Eq. 4, 1: Eq. 5 (the operator D64 belongs to)
  const double *D64;
  const double2 *tw64;
  cudaStream_t st;
  int device;
};

}  // namespace gsm

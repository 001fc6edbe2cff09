// gsm_apply_noalloc: the FP64 matrix-vector product of the plan's operator
// (Eq. 4, or Eq. 5 for an H-field plan) for one point with every temporary in
// one fixed device array, for callers that must not allocate device memory
// during the call (see include/gsm.h).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/gsm.h"
#include "kernels.h"

namespace gsm {
gsm_status plan_full_level(gsm_plan_t *p, PlanView *v);
gsm_status plan_point(gsm_plan_t *p, const gsm_point &pt, const Geo &g, Inst &I);
gsm_status plan_fail(gsm_plan_t *p, gsm_status s, const char *msg);
void plan_count_launches(gsm_plan_t *p, int n);
}  // namespace gsm

using namespace gsm;

// Fixed scratch for the no-allocation product: the intermediate of the three
// passes (3 L_x N_y N_z complex128), the Green denominators (N^3 FP64 and
// FP32) and the instance parameters.  Every GPU that loads the library holds
// it for the life of the process.
static constexpr size_t NOALLOC_SCRATCH_BYTES = 8u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static constexpr int MAX_DEVICES = 64;
static void *g_scratch_ptr[MAX_DEVICES];
static std::mutex g_scratch_mu;

// Device address of the scratch array on `device` (which must be current),
// looked up once per device; the host-side name of the array is only a
// stand-in and must never be handed to a kernel.
static cudaError_t scratch_address(int device, void **out) {
  if (device < 0 || device >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = ptr;
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

static size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

extern "C" gsm_status gsm_apply_noalloc(gsm_plan_t *p, const gsm_point *point, const double *x, double *y) {
  if (!p) return GSM_ERR_ARG;
  if (!point || !x || !y) return plan_fail(p, GSM_ERR_ARG, "gsm_apply_noalloc: NULL argument");
  PlanView v;
  gsm_status s = plan_full_level(p, &v);
  if (s) return s;
  for (int a = 0; a < 3; ++a)
    if (point->n_harm[a] && point->n_harm[a] != v.g.N[a])
      return plan_fail(p, GSM_ERR_ARG, "gsm_apply_noalloc: the point must use the plan's truncation");
  const Geo &g = v.g;
  const size_t need = align256((size_t)g.Tsz * sizeof(double2)) + align256((size_t)g.Nh * sizeof(double)) +
                      align256((size_t)g.Nh * sizeof(float)) + align256(sizeof(Inst));
  if (need > NOALLOC_SCRATCH_BYTES)
    return plan_fail(p, GSM_ERR_ARG,
                     "gsm_apply_noalloc: truncation needs more than the 8 MiB fixed scratch (use gsm_apply)");
  Inst I;
  if ((s = plan_point(p, *point, g, I))) return s;
  if (cudaSetDevice(v.device) != cudaSuccess) {
    cudaGetLastError();
    return plan_fail(p, GSM_ERR_CUDA, "gsm_apply_noalloc: cudaSetDevice failed");
  }
  void *base = nullptr;
  cudaError_t e = scratch_address(v.device, &base);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return plan_fail(p, GSM_ERR_CUDA, "gsm_apply_noalloc: cudaGetSymbolAddress of the scratch array failed");
  }
  char *c = static_cast<char *>(base);
  double2 *T = reinterpret_cast<double2 *>(c);
  c += align256((size_t)g.Tsz * sizeof(double2));
  double *iden64 = reinterpret_cast<double *>(c);
  c += align256((size_t)g.Nh * sizeof(double));
  float *iden32 = reinterpret_cast<float *>(c);
  c += align256((size_t)g.Nh * sizeof(float));
  Inst *inst = reinterpret_cast<Inst *>(c);
  // I lives on the host stack (pageable), so this copy completes before the
  // call returns to the next statement's use of I
  e = cudaMemcpyAsync(inst, &I, sizeof(Inst), cudaMemcpyHostToDevice, v.st);
  if (e == cudaSuccess) e = launch_iden(g, inst, 1, iden64, iden32, v.st);
  if (e == cudaSuccess) {
    MatvecArgs<double> a;
    a.g = g;
    a.B = 1;
    a.X = const_cast<double2 *>(reinterpret_cast<const double2 *>(x));
    a.xstride = g.U;
    a.Y = reinterpret_cast<double2 *>(y);
    a.ystride = g.U;
    a.T = T;
    a.D = v.D64;
    a.inst = inst;
    a.iden = iden64;
    a.tw = v.tw64;
    a.mode = 0;
    a.form = v.form;   // the plan's operator: Eq. 4, or Eq. 5 for an H-field plan
    e = launch_matvec<double>(a, v.st, nullptr);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return plan_fail(p, GSM_ERR_CUDA, cudaGetErrorString(e));
  }
  plan_count_launches(p, 4);
  return GSM_OK;
}

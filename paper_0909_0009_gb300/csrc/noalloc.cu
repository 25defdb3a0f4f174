// fnl_accumulate_noalloc: step (v) (Eq. 5 and Eq. 3) for callers that must not allocate
// device memory.
//
// fnl_accumulate reads the quadrature weights q^X_l[i] = w_i r_i^2 alpha^X_l(r_i) from a
// table that fnl_make_shells allocated.  Some callers cannot make a shells object:
//  - programs whose device memory belongs entirely to another allocator (a framework's
//    caching allocator, a pool sized to the whole GPU), where a stray cudaMalloc fails or
//    fragments that pool;
//  - latency-bound loops, where cudaMalloc and cudaFree may synchronise the device and
//    stall every other stream;
//  - plug-ins that run under a fixed memory budget accounted by their host program.
// This variant of the quadrature kernel keeps its weights in a fixed array compiled into
// the library instead.  The array is device memory of every GPU that loads the library,
// held until the process exits; it needs no allocation call at any time.
#include <algorithm>
#include <mutex>
#include <string>

#include "fnl_internal.cuh"

namespace fnl {

namespace {

// (lmax + 1) * nr weights per component; two components (T, E): 8 MiB in all.
constexpr int64_t kNoallocMaxLNr = FNL_NOALLOC_MAX_LNR;
constexpr int kNoallocMaxDevices = 64;
constexpr int kThreads = 256;

// The scratch: q^T at [0, (lmax+1) nr), q^E right after it.  Every call rewrites the
// (lmax + 1) nr entries of each component that it reads, before reading them, so nothing
// in it has to start at zero and what an earlier call left there is never used.
static __device__ __align__(256) double g_qscratch[2 * kNoallocMaxLNr];

std::mutex g_addr_mutex;
struct ScratchAddr {
  void* ctx = nullptr;   // the CUDA context the address belongs to
  void* addr = nullptr;  // device address of g_qscratch in that context
};
ScratchAddr g_addr[kNoallocMaxDevices];

// The driver's cuCtxGetCurrent (through the runtime's entry-point query, so the library
// needs no link to libcuda): the context that is current on this thread.
void* current_context() {
  typedef int (*CtxGetCurrent)(void**);
  static CtxGetCurrent fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      throw Error(FNL_ECUDA, "fnl_accumulate_noalloc: cuCtxGetCurrent is unavailable");
    }
    fn = (CtxGetCurrent)p;
  }
  void* ctx = nullptr;
  if (fn(&ctx) != 0 || !ctx) throw Error(FNL_ECUDA, "fnl_accumulate_noalloc: no current CUDA context");
  return ctx;
}

// Device address of g_qscratch on device `dev` (the current device).  The address is looked
// up (cudaGetSymbolAddress, which may load the library's device code) on the first call in a
// context and kept with that context: a call in a new context of the same device (after
// cudaDeviceReset, or once the primary context was released and made again) looks it up
// again instead of using an address of memory that no longer exists.  A lookup must not run
// while `st` is being captured into a graph, so such a call is refused with a message.  In
// host code the name g_qscratch stands for a host-side shadow, never for the device memory,
// so only this address reaches a kernel.
double* scratch_address(int dev, cudaStream_t st) {
  if (dev < 0 || dev >= kNoallocMaxDevices)
    throw Error(FNL_EUNSUPPORTED, "fnl_accumulate_noalloc: device ordinal " + std::to_string(dev) +
                                      " is beyond the " + std::to_string(kNoallocMaxDevices) +
                                      " devices this library keeps scratch addresses for");
  void* ctx = current_context();
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  ScratchAddr& a = g_addr[dev];
  if (a.ctx != ctx || !a.addr) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    FNL_CUDA(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      throw Error(FNL_EUNSUPPORTED, "fnl_accumulate_noalloc: the first call in a CUDA context looks up the "
                                    "scratch array's address and cannot run during a stream capture; make one "
                                    "call before the capture begins");
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_qscratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      throw Error(FNL_ECUDA, std::string("fnl_accumulate_noalloc: cudaGetSymbolAddress of the scratch "
                                         "array failed: ") + cudaGetErrorString(e));
    }
    a.ctx = ctx;
    a.addr = p;
  }
  return (double*)a.addr;
}

void check_ptr(const void* p, const char* name, bool nullable, unsigned align, int dev) {
  if (!p) {
    if (!nullable) throw Error(FNL_EINVAL, std::string("fnl_accumulate_noalloc: ") + name + " must not be NULL");
    return;
  }
  if ((uintptr_t)p % align != 0)
    throw Error(FNL_EINVAL, std::string("fnl_accumulate_noalloc: ") + name + " must be " + std::to_string(align) +
                                "-byte aligned");
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    throw Error(FNL_EINVAL, std::string("fnl_accumulate_noalloc: ") + name + " is not a pointer CUDA knows");
  }
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    throw Error(FNL_EINVAL, std::string("fnl_accumulate_noalloc: ") + name + " must be device memory");
  if (attr.type == cudaMemoryTypeDevice && attr.device != dev)
    throw Error(FNL_EINVAL, std::string("fnl_accumulate_noalloc: ") + name +
                                " lives on another device than the current one");
}

// q^X_l[i] = (w_i r_i r_i) alpha^X_l(r_i) into the scratch (the product order of the
// shells object's set-up, so both give the same weights bit for bit).
__global__ void k_weights_noalloc(int L, int nr, const double* __restrict__ r, const double* __restrict__ w,
                                  const double* __restrict__ alphaT, const double* __restrict__ alphaE,
                                  double* __restrict__ q) {
  const int64_t n = (int64_t)(L + 1) * nr;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % nr);
    const double f = w[i] * r[i] * r[i];
    q[e] = f * alphaT[e];
    q[n + e] = f * alphaE[e];
  }
}

__device__ __forceinline__ void lm_of_idx(int64_t idx, int L, int& l, int& m) {
  // entry (m, m) sits at m (2L + 3 - m) / 2; a float estimate of m, corrected exactly
  const float b = 2.0f * L + 3.0f;
  int mm = (int)floorf((b - sqrtf(fmaxf(b * b - 8.0f * (float)idx, 0.0f))) * 0.5f);
  mm = min(max(mm, 0), L);
  while (mm > 0 && alm_idx(mm, mm, L) > idx) --mm;
  while (mm < L && alm_idx(mm + 1, mm + 1, L) <= idx) ++mm;
  m = mm;
  l = (int)(idx - alm_idx(0, mm, L));
}

__device__ __forceinline__ void warp_sum4(double& a, double& b, double& c, double& d) {
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
}

// One warp per (l, m): a^X_L and a^X_NL as FP64 sums over the shells (lane i, i + 32, ...
// then a butterfly), a^X = a^X_L + f_NL a^X_NL.  The weights come from the scratch q.
__global__ void __launch_bounds__(kThreads) k_quadrature_noalloc(int L, int nr, int64_t nalm,
                                                                 const double* __restrict__ q,
                                                                 const double* __restrict__ phiL,
                                                                 const double* __restrict__ phiNL, double fnl,
                                                                 double2* __restrict__ aT, double2* __restrict__ aE,
                                                                 double2* __restrict__ aLT, double2* __restrict__ aLE,
                                                                 double2* __restrict__ aNLT,
                                                                 double2* __restrict__ aNLE) {
  const int64_t idx = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (idx >= nalm) return;
  int l, m;
  lm_of_idx(idx, L, l, m);
  const double* qT = q + (size_t)l * nr;
  const double* qE = q + (size_t)(L + 1) * nr + (size_t)l * nr;
  double lr = 0, li = 0, ler = 0, lei = 0, nr_ = 0, ni = 0, ner = 0, nei = 0;
  if (phiL) {
    const double* row = phiL + (size_t)idx * 2 * nr;
    for (int i = lane; i < nr; i += 32) {
      const double re = row[2 * i], im = row[2 * i + 1];
      lr += qT[i] * re;
      li += qT[i] * im;
      ler += qE[i] * re;
      lei += qE[i] * im;
    }
    warp_sum4(lr, li, ler, lei);
  }
  if (phiNL) {
    const double* row = phiNL + (size_t)idx * 2 * nr;
    for (int i = lane; i < nr; i += 32) {
      const double re = row[2 * i], im = row[2 * i + 1];
      nr_ += qT[i] * re;
      ni += qT[i] * im;
      ner += qE[i] * re;
      nei += qE[i] * im;
    }
    warp_sum4(nr_, ni, ner, nei);
  }
  if (lane) return;
  if (aLT) aLT[idx] = make_double2(lr, li);
  if (aLE) aLE[idx] = make_double2(ler, lei);
  if (aNLT) aNLT[idx] = make_double2(nr_, ni);
  if (aNLE) aNLE[idx] = make_double2(ner, nei);
  if (aT) aT[idx] = make_double2(lr + fnl * nr_, li + fnl * ni);
  if (aE) aE[idx] = make_double2(ler + fnl * ner, lei + fnl * nei);
}

}  // namespace

}  // namespace fnl

extern "C" fnl_status fnl_accumulate_noalloc(int lmax, int nr, const double* r, const double* w,
                                             const double* alphaT, const double* alphaE, const double* phiL,
                                             const double* phiNL, double fnl, double* aT, double* aE, double* aLT,
                                             double* aLE, double* aNLT, double* aNLE, void* stream) {
  using namespace fnl;
  set_last_error("");
  try {
    FNL_REQUIRE(lmax >= 0 && lmax <= 4096, "fnl_accumulate_noalloc: lmax must be in [0, 4096]");
    FNL_REQUIRE(nr >= 1 && nr <= 128, "fnl_accumulate_noalloc: nr must be in [1, 128]");
    const int64_t lnr = (int64_t)(lmax + 1) * nr;
    FNL_REQUIRE(lnr <= kNoallocMaxLNr,
                "fnl_accumulate_noalloc: (lmax + 1) * nr = " + std::to_string(lnr) + " exceeds the fixed scratch of " +
                    std::to_string(kNoallocMaxLNr) +
                    " weights per component; use fnl_accumulate with a shells object for this size");
    int dev = -1;
    FNL_CUDA(cudaGetDevice(&dev));
    for (auto pr : {std::make_pair((const void*)r, "r"), std::make_pair((const void*)w, "w"),
                    std::make_pair((const void*)alphaT, "alphaT"), std::make_pair((const void*)alphaE, "alphaE")})
      check_ptr(pr.first, pr.second, false, 8, dev);
    for (auto pr : {std::make_pair((const void*)phiL, "phiL"), std::make_pair((const void*)phiNL, "phiNL"),
                    std::make_pair((const void*)aT, "aT"), std::make_pair((const void*)aE, "aE"),
                    std::make_pair((const void*)aLT, "aLT"), std::make_pair((const void*)aLE, "aLE"),
                    std::make_pair((const void*)aNLT, "aNLT"), std::make_pair((const void*)aNLE, "aNLE")})
      check_ptr(pr.first, pr.second, true, 16, dev);
    cudaStream_t st = (cudaStream_t)stream;
    double* q = scratch_address(dev, st);
    const int64_t nalm = n_alm(lmax);
    const int wblocks = (int)std::min<int64_t>((lnr + kThreads - 1) / kThreads, 4096);
    k_weights_noalloc<<<wblocks, kThreads, 0, st>>>(lmax, nr, r, w, alphaT, alphaE, q);
    FNL_CUDA(cudaGetLastError());
    const int64_t qblocks = (nalm * 32 + kThreads - 1) / kThreads;
    k_quadrature_noalloc<<<(unsigned)qblocks, kThreads, 0, st>>>(
        lmax, nr, nalm, q, phiL, phiNL, fnl, (double2*)aT, (double2*)aE, (double2*)aLT, (double2*)aLE,
        (double2*)aNLT, (double2*)aNLE);
    FNL_CUDA(cudaGetLastError());
    return FNL_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return FNL_EINVAL;
  } catch (...) {
    set_last_error("unknown error");
    return FNL_EINVAL;
  }
}

// pt_objective_noalloc: the objective of Eq. 2-2-4 for callers that cannot
// allocate device memory.
//
// Some host programs may not allocate GPU memory once they are running, for
// example a station's real-time recording pipeline that reserves the device's
// memory up front in its own pool, or a host framework that forbids driver
// allocations after start-up so its memory use stays fixed. They cannot create
// a pt_ctx (which allocates its buffers) or call pt_objective (which grows
// its scratch on demand). This entry point needs no context: the caller passes
// device buffers for every input and output, and the only scratch is a
// file-scope device array of fixed size that every GPU loading the library
// holds until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cmath>
#include <mutex>

#include "../../include/phasetrack.h"
#include "pt_grid.h"
#include "pt_kernels.cuh"

namespace {

using namespace pt;

constexpr int NOALLOC_MAX_CANDS = PT_NOALLOC_MAX_CANDIDATES;

// Accumulators of up to NOALLOC_MAX_CANDS candidates, then the error word.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[NOALLOC_MAX_CANDS + 32];

std::mutex g_mu;
constexpr int MAX_DEVICES = 64;
unsigned long long* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with that device current, and cached.
int scratch_address(int dev, unsigned long long** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= MAX_DEVICES) return PT_EINVAL;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return PT_ECUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_scratch_addr[dev];
  return PT_OK;
}

// The driver's allocation-range query, looked up once through the runtime (so
// the library does not link the driver library itself). It only reads the
// driver's records of existing allocations and allocates nothing.
typedef CUresult (*AddressRangeFn)(CUdeviceptr* base, size_t* size, CUdeviceptr p);
AddressRangeFn g_address_range = nullptr;
bool g_address_range_looked_up = false;

AddressRangeFn address_range_fn() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_address_range_looked_up) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_address_range = reinterpret_cast<AddressRangeFn>(fn);
    else
      cudaGetLastError();
    g_address_range_looked_up = true;
  }
  return g_address_range;
}

// A caller buffer the kernels may use: device (or managed) memory of device
// `dev`, aligned to `align` bytes, with `bytes` bytes from `p` inside one
// allocation. The kernels read or write exactly that span; a pointer of
// another GPU, an unaligned one or a span past the allocation's end would be
// an invalid access on the device, so each is refused here, before any launch.
bool usable_buffer(const void* p, int dev, size_t align, size_t bytes) {
  cudaPointerAttributes at;
  if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
  if (at.type == cudaMemoryTypeDevice && at.device != dev) return false;
  if (((uintptr_t)p & (align - 1)) != 0) return false;
  const AddressRangeFn range = address_range_fn();
  if (!range) return false;
  CUdeviceptr base = 0;
  size_t size = 0;
  if (range(&base, &size, (CUdeviceptr)(uintptr_t)p) != CUDA_SUCCESS) return false;
  const uintptr_t a = (uintptr_t)p, end = (uintptr_t)base + size;
  return a >= (uintptr_t)base && a <= end && bytes <= end - a;
}

template <int TIER, int CGV>
int launch(const BlockArgs& b, const double* cands, int ncand, unsigned long long* acc, int* err, cudaStream_t s,
           int sms, size_t optin) {
  ObjArgs a{};
  a.b = b;
  a.cands = cands;
  a.ncand = ncand;
  a.cpc = std::min(((ncand + CGV - 1) / CGV) * CGV, NP_MAX);
  const int ny = (ncand + a.cpc - 1) / a.cpc;
  a.tpc = objective_tiles_per_cta(b.ntiles, ny, OBJ_CTAS * sms, [&](int t) {
    return OBJ_CTAS * smem_layout(TIER, a.cpc, t, CGV, b.esize, 0, NT_OBJ).total <= optin;
  });
  const int nx = (int)((b.ntiles + a.tpc - 1) / a.tpc);
  a.acc = acc;
  a.err = err;
  a.timeout_ns = 2000000000ull;
  const SmemLayout S = smem_layout(TIER, a.cpc, a.tpc, CGV, b.esize, 0, NT_OBJ);
  if (S.total > optin) return PT_EINVAL;
  if (cudaFuncSetAttribute(k_objective<TIER, CGV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.total) !=
      cudaSuccess)
    return PT_ECUDA;
  k_objective<TIER, CGV><<<dim3(nx, ny), NT_OBJ, S.total, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? PT_OK : PT_ECUDA;
}

int launch_any(int tier, const BlockArgs& b, const double* cands, int ncand, unsigned long long* acc, int* err,
               cudaStream_t s, int sms, size_t optin) {
  if (tier == PT_TIER_PLAIN) return launch<TIER_PLAIN, 8>(b, cands, ncand, acc, err, s, sms, optin);
  if (tier == PT_TIER_DF32) return launch<TIER_DF32, 8>(b, cands, ncand, acc, err, s, sms, optin);
  if (tier == PT_TIER_F32) return launch<TIER_F32, 8>(b, cands, ncand, acc, err, s, sms, optin);
  const int cg = pick_cg_f64(std::min(ncand, NP_MAX));  // the item width pt_objective uses
  if (cg == 16) return launch<TIER_F64, 16>(b, cands, ncand, acc, err, s, sms, optin);
  if (cg == 8) return launch<TIER_F64, 8>(b, cands, ncand, acc, err, s, sms, optin);
  return launch<TIER_F64, 4>(b, cands, ncand, acc, err, s, sms, optin);
}

}  // namespace

extern "C" int pt_objective_noalloc(const void* samples, int64_t n, int dtype, double scale, double fs, double t0,
                                    double smax, const double* cands, int64_t ncand, double* sse_out, int tier,
                                    void* stream) {
  int esize = 0;
  double bound = 0.0;
  switch (dtype) {
    case PT_I8: esize = 1; bound = 128.0; break;
    case PT_I16: esize = 2; bound = 32768.0; break;
    case PT_F16: esize = 2; bound = 65504.0; break;
    case PT_F32: esize = 4; break;
    case PT_F64: esize = 8; break;
    default: return PT_EINVAL;
  }
  if (n < 1 || n > ((int64_t)1 << 36) || ncand < 1 || ncand > NOALLOC_MAX_CANDS || !(scale > 0.0) ||
      !std::isfinite(scale) || !(fs > 0.0) || !std::isfinite(fs) || !std::isfinite(t0) || tier < PT_TIER_F64 ||
      tier > PT_TIER_F32)
    return PT_EINVAL;
  if (!(smax > 0.0)) {
    if (bound == 0.0) return PT_EINVAL;  // float samples: the caller must bound them
    smax = bound * scale;
  }
  if (!std::isfinite(smax)) return PT_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PT_ECUDA;
  // the staging copies whole 256-sample tiles with 16-byte-aligned bulk copies
  const size_t sample_bytes = (size_t)((n + L - 1) / L) * L * (size_t)esize;
  if (!usable_buffer(samples, dev, 16, sample_bytes) ||
      !usable_buffer(cands, dev, alignof(double), (size_t)ncand * D * sizeof(double)) ||
      !usable_buffer(sse_out, dev, alignof(double), (size_t)ncand * sizeof(double)))
    return PT_EINVAL;
  unsigned long long* scratch = nullptr;
  int rc = scratch_address(dev, &scratch);
  if (rc != PT_OK) return rc;
  int sms = 0, optin = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return PT_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* acc = scratch;
  int* err = reinterpret_cast<int*>(scratch + NOALLOC_MAX_CANDS);
  BlockArgs b{};
  b.samples = samples;
  b.n = n;
  b.ntiles = (n + L - 1) / L;
  b.dtype = dtype;
  b.esize = esize;
  b.scale = scale;
  b.smax = smax;
  b.smax_f = (float)smax;
  b.t0 = t0;
  b.h = 1.0 / fs;
  b.t0sq_2 = t0 * t0 / 2.0;
  b.t0cu_6 = t0 * t0 * t0 / 6.0;
  b.h2_2 = b.h * b.h / 2.0;
  b.h3_6 = b.h * b.h * b.h / 6.0;
  // the array keeps the previous call's contents: clear the accumulators and
  // the error word before every call
  if (cudaMemsetAsync(scratch, 0, (NOALLOC_MAX_CANDS + 1) * sizeof(unsigned long long), s) != cudaSuccess)
    return PT_ECUDA;
  if ((rc = launch_any(tier, b, cands, (int)ncand, acc, err, s, sms, (size_t)optin)) != PT_OK) return rc;
  k_finalize<<<(int)((ncand + 255) / 256), 256, 0, s>>>(cands, (int)ncand, acc, n, (float)smax, sse_out, OBJ_CHI2,
                                                       MODEL_CUBIC, 0.0, 1.0);
  if (cudaGetLastError() != cudaSuccess) return PT_ECUDA;
  int h_err = 0;
  if (cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PT_ECUDA;
  if (h_err == DEV_TIMEOUT) return PT_ETIMEOUT;
  return h_err == DEV_OK ? PT_OK : PT_ECUDA;
}

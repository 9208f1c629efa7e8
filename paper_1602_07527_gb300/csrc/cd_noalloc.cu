// cd_chol_rev_noalloc: the reverse pass for callers that cannot allocate
// device memory.
//
// Some callers may not call cudaMalloc (or any allocating routine) at the
// point where they need a gradient: a custom allocator's own callbacks, or an
// embedding that owns all device memory and forbids the library from taking
// more.  For them this
// entry point runs the same blocked reverse pass as cd_chol_rev, but all of
// its scratch (the inverses of L's diagonal blocks, the solved panel and the
// split-K partial sums) lives in one fixed device array declared below, so
// the call itself allocates nothing and needs no handle.
#include <cuda_runtime.h>

#include <mutex>

#include "cd_internal.h"

namespace cd {
size_t rev_scratch_need(int n, int nb);
int rev_in_scratch(int n, const double *L, long long ldl, double *Abar, long long lda, int nb, int out,
                   void *scratch, size_t scratch_bytes, int num_sms, cudaStream_t s);
}  // namespace cd

namespace {

// 8 MiB, held by every GPU that loads the library until the process exits.
constexpr size_t kScratchBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices];  // device address of g_scratch, per device
int g_sms[kMaxDevices];

// Once per device, with that device current: look up the device address of
// the scratch array (the host-side name g_scratch is only a stand-in and must
// never be passed to a kernel) and prepare the tile kernels.
int setup(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_ptr[dev]) return CD_OK;
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return CD_ECUDA;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CD_ECUDA;
  if (cd::tile_kernels_init() != cudaSuccess) return CD_ECUDA;
  g_sms[dev] = sms;
  g_ptr[dev] = p;
  return CD_OK;
}

}  // namespace

extern "C" int cd_chol_rev_noalloc(int n, const double *L, long long ldl, double *Abar, long long lda, int nb,
                                   int out, void *stream) {
  if (n < 0 || nb < 0 || nb > CD_NOALLOC_MAX_NB || (out != CD_OUT_TRIL && out != CD_OUT_SYM)) return CD_EINVAL;
  if (n > CD_NOALLOC_MAX_N) return CD_ESCRATCH;
  if (n == 0) return CD_OK;
  if (!L || !Abar || ldl < n || lda < n) return CD_EINVAL;
  if (nb == 0) nb = n >= 1024 ? 128 : 64;
  if (cd::rev_scratch_need(n, nb) > kScratchBytes) return CD_ESCRATCH;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CD_ECUDA;
  const int rc = setup(dev);
  if (rc != CD_OK) return rc;
  return cd::rev_in_scratch(n, L, ldl, Abar, lda, nb, out, g_ptr[dev], kScratchBytes, g_sms[dev],
                            (cudaStream_t)stream);
}

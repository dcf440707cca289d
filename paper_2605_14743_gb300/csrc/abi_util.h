// abi_util.h -- error reporting and device queries shared by the C-ABI translation units
// (abi.cu: counting, chain and host-query entry points; abi_analysis.cu: the analyses built on
// an estimated chain).
#pragma once

#include <cstdarg>
#include <cstdio>
#include <exception>
#include <new>
#include <string>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "afc.h"

namespace afc {

// An NVTX range around a C-ABI call (shows up in Nsight timelines; a no-op without a tool).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// The calling thread's last error message (afc_last_error) and the helpers that set it.
std::string &abi_error_text();
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define AFC_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e__ = (call);                            \
    if (e__ != cudaSuccess) return cuda_fail(e__, #call); \
  } while (0)

struct DevInfo {
  int sms = 0, smem_optin = 0;
};
DevInfo dev_info();

// The chain parameters every analysis entry point needs: n >= 1, R > 0, alpha in [0, 1] (the
// absorption probability of Sec. 4) and the floor eta in (0, 1) (Sec. 8.2 stabilisation).
inline int chain_params_check(const afc_chain *ch) {
  if (ch->n < 1) return fail(AFC_EINVAL, "n must be >= 1");
  if (ch->realizations == 0) return fail(AFC_EINVAL, "realizations must be > 0");
  if (!(ch->alpha >= 0.0 && ch->alpha <= 1.0)) return fail(AFC_EINVAL, "alpha outside [0, 1]");
  if (!(ch->absorb_floor > 0.0 && ch->absorb_floor < 1.0))
    return fail(AFC_EINVAL, "absorb_floor outside (0, 1)");
  return AFC_OK;
}

// Host entry points that allocate run their body through this: a C caller gets AFC_ENOMEM
// (or AFC_EDEVICE for anything else) instead of an exception crossing the C ABI.
template <typename Fn>
int guarded(const char *what, Fn &&fn) {
  try {
    return fn();
  } catch (const std::bad_alloc &) {
    return fail(AFC_ENOMEM, "%s: host allocation failed", what);
  } catch (const std::exception &e) {
    return fail(AFC_EDEVICE, "%s: %s", what, e.what());
  }
}

}  // namespace afc

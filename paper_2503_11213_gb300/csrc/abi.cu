// Library-wide C ABI helpers: status strings, version, last CUDA error.
#include "common.cuh"

namespace sd {
namespace {
thread_local int t_last_cuda_error = 0;
}
void set_cuda_error(cudaError_t e) { t_last_cuda_error = (int)e; }
}  // namespace sd

extern "C" {

const char* sd_status_string(sd_status s) {
  switch (s) {
    case SD_OK: return "ok";
    case SD_ERR_ARG: return "invalid argument";
    case SD_ERR_LENS: return "invalid lens prescription";
    case SD_ERR_UNSUPPORTED: return "unsupported configuration";
    case SD_ERR_CUDA: return "CUDA runtime error";
    case SD_ERR_CAPACITY: return "library table full";
    default: return "unknown status";
  }
}

int sd_last_cuda_error(void) { return sd::t_last_cuda_error; }

int sd_version(void) { return 100; }

}  // extern "C"

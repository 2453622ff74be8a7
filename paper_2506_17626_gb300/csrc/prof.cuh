// prof.cuh -- scope guard that brackets a kernel launch with CUDA events when
// profiling is enabled (rfm_profile_enable); a no-op otherwise.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rfm {
class ProfScope {
  public:
    ProfScope(const char *name, cudaStream_t st);
    ~ProfScope();

  private:
    const char *name_;
    cudaStream_t st_;
    void *a_ = nullptr, *b_ = nullptr;
    bool on_;
};
void prof_enable(bool on);
void prof_reset();
int prof_read(const char **names, int64_t *launches, double *ms, int max);
}  // namespace rfm

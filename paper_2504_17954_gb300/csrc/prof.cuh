// RAII bracket of one kernel launch for the opt-in per-kernel timer (see prof.cu).
#pragma once

#include <cuda_runtime.h>

namespace ivrgs {

class ProfScope {
  public:
    ProfScope(const char* name, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    const char* name_;
    cudaStream_t s_;
    cudaEvent_t a_;
};

}  // namespace ivrgs

#define IVRGS_CAT2(a, b) a##b
#define IVRGS_CAT(a, b) IVRGS_CAT2(a, b)
#define IVRGS_PROF(name, stream) ::ivrgs::ProfScope IVRGS_CAT(ivrgs_prof_scope_, __LINE__)(name, stream)

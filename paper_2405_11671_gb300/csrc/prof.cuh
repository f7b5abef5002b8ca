// prof.cuh -- launch counter and event-bracketed kernel timing (prof.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace byo {

void note_launch(uint64_t k = 1);
bool profiling_on();

// Records an event on `s` at construction and at destruction when profiling
// is on; the pair is attributed to `name` (a string literal).
class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t s);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  void* a_;
};

}  // namespace byo

// Launch accounting: wrap every kernel launch as
//   { LaunchScope ls(stream, "k_name"); k_name<<<..., stream>>>(...); }
#pragma once

#include <cuda_runtime.h>

namespace mpap {

class LaunchScope {
 public:
  LaunchScope(cudaStream_t st, const char* name);
  ~LaunchScope();
  LaunchScope(const LaunchScope&) = delete;
  LaunchScope& operator=(const LaunchScope&) = delete;

 private:
  cudaStream_t st_;
  const char* name_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

}  // namespace mpap

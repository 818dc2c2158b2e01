// kernels.cuh -- launchers of the device kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace ubs {

// the views that render one scene, by index into the view table
struct ViewList {
  int32_t n;
  int16_t idx[kMaxViews];
};

cudaError_t launch_preprocess(const SceneDev& sc, const ViewList& vl, const ViewDev* views, const CfgDev& cfg,
                              const Layout& L, char* ws, cudaStream_t st);

// scan/sort/emit/ranges; leaves the sorted instance records in the buffer
// reported by sorted_instances()
cudaError_t launch_bin_sort(const Layout& L, const CfgDev& cfg, char* ws, cudaStream_t st);
const uint32_t* sorted_instances(const Layout& L, const char* ws);

cudaError_t launch_render_fwd(const Layout& L, const CfgDev& cfg, char* ws, float* image, cudaStream_t st);
cudaError_t launch_render_bwd(const Layout& L, const CfgDev& cfg, char* ws, const float* dL_dimage, cudaStream_t st);
cudaError_t launch_prim_backward(const SceneDev& sc, const SceneGradDev& g, const ViewList& vl, const ViewDev* views,
                                 const CfgDev& cfg, const Layout& L, char* ws, cudaStream_t st);

}  // namespace ubs

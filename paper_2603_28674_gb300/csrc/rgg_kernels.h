// Host-visible launch interface of the RGG kernels (internal to librgg.so).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "rgg_device.cuh"

namespace rgg {

constexpr int kNumStages = 3;          // smem ring depth of the streaming pipeline
constexpr int kStageBytes = 48 * 1024; // bytes per stage (records + tile metadata)
constexpr int kMaxBuildLinks = 32;
constexpr uint32_t kMaxUpdateBoxes = 256;  // poses carried by value per update launch

struct BuildParams {
  uint32_t L, K;
  double a[kMaxBuildLinks], alpha[kMaxBuildLinks], d[kMaxBuildLinks], radius[kMaxBuildLinks];
  const double* qa;
  const double* qb;
  const uint64_t* soff;
  float* inner;
  float* outer;
  uint64_t in_stride, out_stride;
  uint64_t n_edges;
};

struct BoxUpdateParams {
  uint32_t n;
  uint32_t ids[kMaxUpdateBoxes];
  float pose[kMaxUpdateBoxes][15];
  const float* dev_pose;  // if non-null, poses are read from device memory
  float* table;           // [M][16]
};

struct BoxPrepJob {
  const float* table;
  float* out;             // [C][24]
  uint32_t C;
  uint32_t ids[kBoxesPerPass];
};

struct BoxPrepParams {
  BoxPrepJob job[kMaxJobs];
  uint32_t njobs;
};

struct ClassifyLaunch {
  uint32_t grid;
  uint32_t consumer_warps;
  uint32_t tw_cap;   // max intervals per tile over the launch's jobs
  uint32_t acc_cap;  // max local edges per tile over the launch's jobs
};

size_t classify_smem_bytes(uint32_t tw_cap, uint32_t acc_cap);

cudaError_t launch_count_samples(const double* qa, const double* qb, uint64_t n_edges, uint32_t L,
                                 double step, uint64_t* counts, int* bad, cudaStream_t s);
cudaError_t launch_build_records(const BuildParams& p, int num_sms, cudaStream_t s);
cudaError_t launch_tile_edge(const uint64_t* soff, uint64_t n_edges, uint32_t L, uint32_t S,
                             uint64_t n_tiles, uint32_t* out, cudaStream_t s);
cudaError_t launch_box_update(const BoxUpdateParams& p, cudaStream_t s);
cudaError_t launch_box_prep(const BoxPrepParams& p, cudaStream_t s);
cudaError_t launch_classify_single(const ClassifyParams<1>& p, const ClassifyLaunch& lc,
                                   cudaStream_t s);
cudaError_t launch_classify_batched(const ClassifyParams<kMaxJobs>& p, const ClassifyLaunch& lc,
                                    cudaStream_t s);

}  // namespace rgg

// Internal launch interface between the C ABI (pg_api.cu) and the kernels
// (pg_kernels.cu). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pg_device.cuh"

namespace pgk {

struct SamplePlanes {
    float *wx, *wy, *wz, *radiance, *pdf, *mis, *estimate;
    uint8_t* strategy;
};

// Every launcher returns cudaGetLastError() of its launch.
cudaError_t launch_init(int dt, const Params& P, void* gam, float init_pi, cudaStream_t st);
cudaError_t launch_frame(int dt, const Params& P, const void* gin, void* gout, const float4* g0,
                         const float4* g1, const float4* g0p, float* img, uint32_t frame, int* err,
                         cudaStream_t st);
// neighbour-VPL reuse: the path-tracing pass (writes the VPL buffer and each pixel's handover
// record {Z, reprojection outcome}) and the training pass (reads both)
cudaError_t launch_pt(int dt, const Params& P, const void* gin, const float4* g0, const float4* g1,
                      const float4* g0p, float* img, uint32_t frame, float4* vpl, float* pb_src, float2* hand,
                      int* err, cudaStream_t st);
cudaError_t launch_train(int dt, const Params& P, const void* gin, void* gout, const float4* g0, const float4* g1,
                         const float4* g0p, uint32_t frame, const float4* vpl, const float* pb_src, const float2* hand,
                         int* err, cudaStream_t st);
cudaError_t launch_reproject(int dt, const Params& P, const void* gin, float4* work, const float4* g0,
                             const float4* g1, const float4* g0p, uint8_t* accept, int* err, cudaStream_t st);
cudaError_t launch_sample(int dt, const Params& P, const float4* work, const float4* g0, const float4* g1,
                          uint32_t frame, SamplePlanes out, float* img, cudaStream_t st);
cudaError_t launch_update(int dt, const Params& P, const float4* work, const float4* g0, const float4* g1,
                          SamplePlanes in, void* gout, int* err, cudaStream_t st);
cudaError_t launch_eval(int dt, const Params& P, const void* src, bool src_is_work, const float4* g0,
                        const float4* g1, int n_dirs, const float* dirs, float* out, cudaStream_t st);
cudaError_t launch_to_f32(int dt, const Params& P, const void* src, bool src_is_work, float4* dst,
                          cudaStream_t st);
cudaError_t launch_from_f32(int dt, const Params& P, const float4* src, void* dst, cudaStream_t st);

cudaError_t launch_grad(int dt, const Params& P, const void* gam, const float* theta, const float4* g0,
                        const float4* g1, uint32_t frame, int n, float* loss, float* grad, cudaStream_t st);
// Adam: binary32 moments as [6][H*W] planes m and v; BF16 moments as one
// 24-byte record per pixel {m_0..m_5, v_0..v_5} (rec), converted to and from
// binary32 planes by the rec_get / rec_set launchers
cudaError_t launch_adam(int dt, const Params& P, void* gam, const float* grad, float* m, float* v, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st);
cudaError_t launch_adam_bf16(int dt, const Params& P, void* gam, const float* grad, void* rec, float lr, float b1,
                             float b2, float eps, float c1, float c2, uint32_t step, cudaStream_t st);
cudaError_t launch_adam_rec_get(const Params& P, const void* rec, float* m, float* v, cudaStream_t st);
cudaError_t launch_adam_rec_set(const Params& P, const float* m, const float* v, void* rec, cudaStream_t st);
cudaError_t launch_theta_get(int dt, const Params& P, const void* gam, float* theta, cudaStream_t st);
cudaError_t launch_theta_set(int dt, const Params& P, void* gam, const float* theta, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int64_t n, uint32_t* out, bool curand,
                          cudaStream_t st);

}  // namespace pgk

// A whole staged frame for callers that cannot allocate device memory.
//
// Some hosts cannot call cudaMalloc at all: an engine whose device memory
// is carved out once at start-up by its own allocator, a plug-in running
// inside such an engine, or code that must not allocate while a frame is in
// flight. pg_frame_noalloc runs the three staged kernels (reprojection,
// sampling, training) without a context and without any allocation: the
// caller passes Gamma in and out, the G-buffer, the sample records and the
// image, and the only intermediate buffer, the binary32 work copy of Gamma
// between the reprojection and the training step, lives in a file-scope
// device array of fixed size.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/pg.h"
#include "pg_launch.h"
#include "pg_params.h"

namespace {

// The fixed scratch: 2 float4 per pixel for at most 2^18 pixels (8 MiB),
// plus the word the training kernel raises on a non-finite Gamma. Every GPU
// that loads the library holds this memory until the process exits.
constexpr size_t kStaticMaxPixels = size_t(1) << 18;
__device__ __align__(256) float4 g_static_work[2 * kStaticMaxPixels];
__device__ __align__(256) int g_static_flag[64];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
float4* g_work_addr[kMaxDevices] = {};
int* g_flag_addr[kMaxDevices] = {};

// Device addresses of the scratch on the current device, looked up once per
// device and kept for the life of the process (a cudaDeviceReset of that
// device would leave them stale; pg.h says so). In host code the names
// g_static_work / g_static_flag denote host stand-ins, not device memory, so
// only these addresses may reach a kernel.
pg_status static_scratch(float4** work, int** flag) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PG_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_work_addr[dev]) {
        void *w = nullptr, *f = nullptr;
        if (cudaGetSymbolAddress(&w, g_static_work) != cudaSuccess) return PG_ERR_CUDA;
        if (cudaGetSymbolAddress(&f, g_static_flag) != cudaSuccess) return PG_ERR_CUDA;
        g_work_addr[dev] = static_cast<float4*>(w);
        g_flag_addr[dev] = static_cast<int*>(f);
    }
    *work = g_work_addr[dev];
    *flag = g_flag_addr[dev];
    return PG_OK;
}

bool overlap(const void* a, size_t na, const void* b, size_t nb) {
    const char *pa = static_cast<const char*>(a), *pb = static_cast<const char*>(b);
    return pa < pb + nb && pb < pa + na;
}

}  // namespace

extern "C" pg_status pg_frame_noalloc(const pg_config* cfg, const pg_gbuffer* cur, const float* d_g0_prev,
                                      const pg_field* field, uint32_t frame, const void* d_gamma_in,
                                      void* d_gamma_out, const pg_samples* d_samples, float* d_img,
                                      void* stream) {
    std::string why;
    if (!cfg || pgk::check_config(cfg, why) != PG_OK) return PG_ERR_ARG;
    if (cfg->reuse_radius > 0) {
        std::fprintf(stderr, "pg_frame_noalloc: neighbour reuse needs the VPL buffer of a context (pg_frame)\n");
        return PG_ERR_ARG;
    }
    const size_t hw = (size_t)cfg->width * cfg->height;
    if (hw > kStaticMaxPixels) {
        std::fprintf(stderr, "pg_frame_noalloc: %d x %d = %zu pixels exceeds the fixed scratch of %zu pixels\n",
                     cfg->width, cfg->height, hw, kStaticMaxPixels);
        return PG_ERR_ARG;
    }
    if (!cur || !cur->g0 || !cur->g1 || !pgk::aligned16(cur->g0) || !pgk::aligned16(cur->g1)) return PG_ERR_ARG;
    if (!d_g0_prev || !pgk::aligned16(d_g0_prev)) return PG_ERR_ARG;
    if (!d_gamma_in || !d_gamma_out || !pgk::aligned16(d_gamma_in) || !pgk::aligned16(d_gamma_out))
        return PG_ERR_ARG;
    const size_t gbytes = hw * (cfg->gamma_dtype == PG_F32 ? 32 : 16);
    if (d_gamma_in != d_gamma_out && overlap(d_gamma_in, gbytes, d_gamma_out, gbytes)) return PG_ERR_ARG;
    if (!d_samples || !d_samples->wx || !d_samples->wy || !d_samples->wz || !d_samples->radiance ||
        !d_samples->strategy)
        return PG_ERR_ARG;

    pgk::Params P;
    pgk::config_params(*cfg, P);
    if (pgk::camera_params(cur->camera, P, why) != PG_OK) return PG_ERR_ARG;
    if (pgk::field_params(field, P, why) != PG_OK) return PG_ERR_ARG;

    float4* work = nullptr;
    int* flag = nullptr;
    if (static_scratch(&work, &flag) != PG_OK) return PG_ERR_CUDA;

    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int dt = cfg->gamma_dtype;
    const float4* g0 = reinterpret_cast<const float4*>(cur->g0);
    const float4* g1 = reinterpret_cast<const float4*>(cur->g1);
    pgk::SamplePlanes s{d_samples->wx,  d_samples->wy,       d_samples->wz,       d_samples->radiance,
                        d_samples->pdf, d_samples->mis,      d_samples->estimate, d_samples->strategy};
    // the flag word keeps the previous call's value: clear it first
    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return PG_ERR_CUDA;
    if (pgk::launch_reproject(dt, P, d_gamma_in, work, g0, g1, reinterpret_cast<const float4*>(d_g0_prev), nullptr,
                              flag, st) != cudaSuccess)
        return PG_ERR_CUDA;
    if (pgk::launch_sample(dt, P, work, g0, g1, frame, s, d_img, st) != cudaSuccess) return PG_ERR_CUDA;
    P.sr_frame = frame;
    if (pgk::launch_update(dt, P, work, g0, g1, s, d_gamma_out, flag, st) != cudaSuccess) return PG_ERR_CUDA;
    return PG_OK;
}

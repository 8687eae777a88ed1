// Allocation-free steady-state residual for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: an application that hands the library a fixed
// device-memory arena and forbids allocations after start-up, or a real-time loop in which an
// allocation would stall (cudaMalloc may synchronise the device).  This file gives them one
// entry point, lbm_residual_noalloc, that computes the same relative change of the velocity
// and temperature fields as lbm_residual from fields the caller already holds, and keeps its
// per-block partial sums in a fixed, file-scope device array instead.
//
// The array lives for as long as the library is loaded, on every GPU that loads it.  Every
// call shares it and it keeps the last call's contents; each call writes every slot it
// reads before reading it, so nothing has to be cleared.  Calls whose kernels overlap on the
// GPU (two streams, or two host threads) race on the array: serialise them.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/lbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSitesPerBlock = 4096;  // 16 sites per thread
constexpr int kMaxBlocks = LBM_NOALLOC_MAX_SITES / kSitesPerBlock;
constexpr int kVals = 5;  // sum |du|^2, sum |u|^2, sum dT^2, sum T^2, non-finite count
constexpr int kMaxDevices = 64;

static_assert(LBM_NOALLOC_MAX_SITES % kSitesPerBlock == 0, "whole blocks");

// Partial sums of one call: kVals per block, 8192 blocks at most (320 KiB).
static __device__ __align__(256) double g_residual_scratch[kMaxBlocks * kVals];

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// One block per 4096 sites; block b writes slots [kVals*b, kVals*b + kVals).
__global__ void __launch_bounds__(kThreads)
    residual_partials_kernel(const float* __restrict__ u, const float* __restrict__ T,
                             const float* __restrict__ up, const float* __restrict__ Tp,
                             long long ns, double* __restrict__ scratch) {
    double v[kVals] = {0.0, 0.0, 0.0, 0.0, 0.0};
    long long base = (long long)blockIdx.x * kSitesPerBlock;
    long long end = base + kSitesPerBlock < ns ? base + kSitesPerBlock : ns;
    for (long long s = base + threadIdx.x; s < end; s += kThreads) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double x = u[a * ns + s], d = x - (double)up[a * ns + s];
            v[0] += d * d;
            v[1] += x * x;
            if (!isfinite(x)) v[4] += 1.0;
        }
        double t = T[s], dt = t - (double)Tp[s];
        v[2] += dt * dt;
        v[3] += t * t;
        if (!isfinite(t)) v[4] += 1.0;
    }
    __shared__ double sh[kVals][kThreads / 32];
#pragma unroll
    for (int k = 0; k < kVals; ++k) {
        double x = warp_sum(v[k]);
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int k = 0; k < kVals; ++k) {
            double x = warp_sum(threadIdx.x < kThreads / 32 ? sh[k][threadIdx.x] : 0.0);
            if (threadIdx.x == 0) scratch[kVals * blockIdx.x + k] = x;
        }
    }
}

// Sums the partials of `nblocks` blocks and writes (r_u, r_T, non-finite count) to out.
__global__ void __launch_bounds__(kThreads)
    residual_finish_kernel(const double* __restrict__ scratch, int nblocks,
                           double* __restrict__ out) {
    double v[kVals] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kThreads)
#pragma unroll
        for (int k = 0; k < kVals; ++k) v[k] += scratch[kVals * b + k];
    __shared__ double sh[kVals][kThreads / 32];
#pragma unroll
    for (int k = 0; k < kVals; ++k) {
        double x = warp_sum(v[k]);
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double t[kVals];
#pragma unroll
        for (int k = 0; k < kVals; ++k)
            t[k] = warp_sum(threadIdx.x < kThreads / 32 ? sh[k][threadIdx.x] : 0.0);
        if (threadIdx.x == 0) {
            if (t[4] > 0.0) {  // a non-finite value: no residual, and never below a tolerance
                out[0] = nan("");
                out[1] = nan("");
            } else {
                out[0] = t[1] > 0.0 ? sqrt(t[0] / t[1]) : (t[0] > 0.0 ? HUGE_VAL : 0.0);
                out[1] = t[3] > 0.0 ? sqrt(t[2] / t[3]) : (t[2] > 0.0 ? HUGE_VAL : 0.0);
            }
            out[2] = t[4];
        }
    }
}

// Device address of the scratch array, looked up once per device by the first call made on
// that device; that first call belongs before any stream capture begins.
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

cudaError_t scratch_for_device(int dev, double** ptr) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        // With `dev` current: the host-side name of the array is only a stand-in, the kernels
        // need the device address.
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *ptr = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Makes `dev` the calling thread's current device for the lifetime of the guard and restores
// the device that was current before on every exit.
class DeviceGuard {
  public:
    cudaError_t enter(int dev) {
        cudaError_t e = cudaGetDevice(&prev_);
        if (e != cudaSuccess) return e;
        have_prev_ = true;
        return prev_ == dev ? cudaSuccess : cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int now = -1;
        if (have_prev_ && cudaGetDevice(&now) == cudaSuccess && now != prev_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0;
    bool have_prev_ = false;
};

}  // namespace

extern "C" lbm_status lbm_residual_noalloc(const float* u, const float* T, const float* u_prev,
                                           const float* T_prev, long long ns, double* out,
                                           void* stream) {
    if (!u || !T || !u_prev || !T_prev || !out) return LBM_EINVAL;
    if (ns < 1 || ns > LBM_NOALLOC_MAX_SITES) return LBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    cudaError_t e = st ? cudaStreamGetDevice(st, &dev) : cudaGetDevice(&dev);
    if (e != cudaSuccess) return LBM_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return LBM_EINVAL;
    DeviceGuard guard;  // the caller's current device is back in place on every return
    if (guard.enter(dev) != cudaSuccess) return LBM_ECUDA;
    double* scratch = nullptr;
    if (scratch_for_device(dev, &scratch) != cudaSuccess) return LBM_ECUDA;
    const int nblocks = (int)((ns + kSitesPerBlock - 1) / kSitesPerBlock);
    // each launch is checked through its own return code, so an error left on the thread by
    // an earlier, unrelated call is neither reported as this call's nor cleared
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cfg.gridDim = dim3(nblocks);
    if (cudaLaunchKernelEx(&cfg, residual_partials_kernel, u, T, u_prev, T_prev, ns, scratch) !=
        cudaSuccess)
        return LBM_ECUDA;
    cfg.gridDim = dim3(1);
    if (cudaLaunchKernelEx(&cfg, residual_finish_kernel, (const double*)scratch, nblocks, out) !=
        cudaSuccess)
        return LBM_ECUDA;
    return LBM_OK;
}

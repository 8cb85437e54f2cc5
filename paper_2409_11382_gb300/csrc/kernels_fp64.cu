// FP64 instantiation of the kernels (the FP64 path, and the coarsest level of
// the FP32 path).  Compiled with --fmad=false so that no fused multiply-add
// changes the rounding.
#include "instantiate.h"

BIOT_SWEEP_MOM(double, double)
BIOT_SEGMENT(double)
BIOT_FIELDS(double)

// Stopping test of one V-cycle (tolerance mode, inside a CUDA graph):
// converged when max|g - ELASTIC_STEP(g)| <= tol * max(1, max|g|); the loop also
// stops at ne_max V-cycles or at a non-finite residual.  Sets the WHILE node's
// condition and the per-instance counters the host reads once per biot_step.
__global__ void k_stop_test(const biot::StopArgs a)
{
    biot::StopState &s = *a.st;
    if (a.first) s.ne = 0;
    s.ne += 1;
    s.total += 1;
    const double res = __longlong_as_double((long long)a.resmax[0]);
    const double gn = __longlong_as_double((long long)a.resmax[1]);
    s.last_res = res;
    s.last_gn = gn;
    const bool finite = (res == res) && res <= 1.7976931348623157e308;
    const bool conv = finite && res <= a.tol * (gn > 1.0 ? gn : 1.0);
    const bool cont = finite && !conv && s.ne < a.ne_max;
    if (!cont) {
        s.last_ne = s.ne;
        if (!finite) s.diverged = 1;
        else if (!conv) s.notconv += 1;
    }
    cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, cont ? 1u : 0u);
}

cudaError_t biot::launch_stop_test(const biot::StopArgs &a, cudaStream_t s)
{
    k_stop_test<<<1, 1, 0, s>>>(a);
    return cudaGetLastError();
}

// State hand-over from an FP64 instance to an FP32 one (see NarrowArgs).
__global__ void __launch_bounds__(256) k_narrow_state(const biot::NarrowArgs a)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.np; i += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const double v = a.g64[k * a.np + i];
            const float hi = (float)v;
            a.g32[k * a.np + i] = hi;
            if (k < 2) a.glo32[k * a.np + i] = (float)(v - (double)hi);
        }
#pragma unroll
        for (int k = 0; k < 9; k++) a.f32[k * a.np + i] = (float)a.f64[k * a.np + i];
#pragma unroll
        for (int k = 0; k < 2; k++) a.ft32[k * a.np + i] = (float)a.ft64[k * a.np + i];
    }
}

cudaError_t biot::launch_narrow_state(const biot::NarrowArgs &a, cudaStream_t s)
{
    if (a.np == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((a.np + 255) / 256 < 65536 ? (a.np + 255) / 256 : 65536);
    k_narrow_state<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// The deviation store encoded from FP32 planes 2-4 (see DevEncodeArgs).
__global__ void __launch_bounds__(256) k_dev_encode(const biot::DevEncodeArgs a)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.np; i += (size_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float v = a.g[(2 + k) * a.np + i] * a.dsc;
            if (a.dev == 1) biot::dev_store<1>(a.gd, k * a.np + i, v);
            else biot::dev_store<2>(a.gd, k * a.np + i, v);
        }
    }
}

cudaError_t biot::launch_dev_encode(const biot::DevEncodeArgs &a, cudaStream_t s)
{
    if (a.np == 0) return cudaSuccess;
    if (a.dev != 1 && a.dev != 2) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)((a.np + 255) / 256 < 65536 ? (a.np + 255) / 256 : 65536);
    k_dev_encode<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

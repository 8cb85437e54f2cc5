// sweep_batch.cuh -- the work-list forms of the elastic sweeps, used by batches
// of instances: one launch runs strips (or tiles) of the sweeps of many
// instances and multigrid levels of one storage kind.  The per-cell code is the
// single-instance sweep of sweep_mom.cuh; only the mapping of CTAs to work items
// and the source of the arguments differ.
#pragma once
#include "sweep_mom.cuh"

namespace biot {

// The job of work item b of a batched launch (binary search over the item
// ranges; the same for every thread of a CTA).
template <typename T, typename TC>
__device__ __forceinline__ int batch_job(const BatchParams<T, TC> &P, int b)
{
    int lo = 0, hi = P.njobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Batched form: CTA b processes work item b, a strip of the sweep of its job (the
// jobs of one launch may belong to different instances and different multigrid
// levels of one storage kind).  The arguments are read from the launch's
// parameter block, which lives in constant memory.
template <typename T, typename TC, int NT, int CPT, int KIND, bool LO, bool RESTRICT>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 896 / (NT * CPT) : 1)
    k_sweep_batch(const __grid_constant__ BatchParams<T, TC> P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3][NT / 32];
    const int j = batch_job(P, blockIdx.x);
    const int local = blockIdx.x - P.start[j], sx = P.sx[j];
    sweep_strip_any<T, TC, NT, CPT, KIND, LO, RESTRICT, FETCH_DYN>(P.job[j], local % sx, local / sx, P.ty[j], smem_raw, red);
}

// Batched form: CTA b processes work item b, a tile of the sweep of its job.
template <typename T, typename TC, int TX, int TY, int KIND, bool LO, bool RESTRICT>
__global__ void __launch_bounds__(TileShape<TX, TY>::NT)
    k_sweep_tile_batch(const __grid_constant__ BatchParams<T, TC> P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3][TileShape<TX, TY>::NT / 32];
    const int j = batch_job(P, blockIdx.x);
    const int local = blockIdx.x - P.start[j], sx = P.sx[j];
    tile_body<T, TC, TX, TY, KIND, LO, RESTRICT>(P.job[j], local % sx, local / sx, smem_raw, red);
}

template <typename T, typename TC, int KIND, bool LO, bool RESTRICT>
cudaError_t launch_tile_batch(const BatchParams<T, TC> &P, cudaStream_t s)
{
    constexpr int TX = TileFor<T>::X, TY = TileFor<T>::Y;
    constexpr size_t smem = tile_smem_bytes<T, TX, TY, KIND, LO>();
    auto kern = k_sweep_tile_batch<T, TC, TX, TY, KIND, LO, RESTRICT>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int n = P.start[P.njobs];
    if (n <= 0) return cudaSuccess;
    kern<<<n, TileShape<TX, TY>::NT, smem, s>>>(P);
    return cudaGetLastError();
}

// The strip form's kernel attributes and resident CTAs per device (set up on
// first use).
// Strip shape of the batched kernel: 128 threads, one cell of a row each
// (measured on the 64-instance workload: 7.28 ms per step, against 7.62 ms with
// the single-instance kernel's 192 threads).
constexpr int BATCH_NT = 128;
static_assert(BATCH_NT - 4 == BATCH_STRIP_COLS, "strip geometry shared with the host planner");

template <typename T, typename TC, int KIND, bool LO, bool RESTRICT>
struct BatchKernel {
    static constexpr size_t smem = rows_smem_bytes<T, KIND, LO, BATCH_NT>();
    static int slots()
    {
        static int n = 0;
        if (!n) {
            auto k = k_sweep_batch<T, TC, BATCH_NT, 1, KIND, LO, RESTRICT>;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
            int dev = 0, sms = 0, per_sm = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) return 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BATCH_NT, smem) != cudaSuccess) return 0;
            n = sms * (per_sm > 0 ? per_sm : 1);
        }
        return n;
    }
};

template <typename T, typename TC, int KIND, bool LO, bool RESTRICT>
cudaError_t launch_batch_v(const BatchParams<T, TC> &P, cudaStream_t s)
{
    using BK = BatchKernel<T, TC, KIND, LO, RESTRICT>;
    const int n = P.start[P.njobs];
    if (n <= 0) return cudaSuccess;
    if (!BK::slots()) return cudaErrorInvalidConfiguration;
    k_sweep_batch<T, TC, BATCH_NT, 1, KIND, LO, RESTRICT><<<n, BATCH_NT, BK::smem, s>>>(P);
    return cudaGetLastError();
}

template <typename T, typename TC, int KIND, bool LO, bool RS>
struct BatchRun {
    static cudaError_t run(bool tile, const BatchParams<T, TC> &P, cudaStream_t s)
    {
        return tile ? launch_tile_batch<T, TC, KIND, LO, RS>(P, s) : launch_batch_v<T, TC, KIND, LO, RS>(P, s);
    }
};
template <typename T, typename TC, int KIND, bool LO, bool RS>
struct SlotsRun {
    static int run() { return BatchKernel<T, TC, KIND, LO, RS>::slots(); }
};

template <typename T, typename TC>
cudaError_t launch_sweep_batch_impl(int v, const BatchParams<T, TC> &P, cudaStream_t s)
{
    return dispatch_kind<T, TC, BatchRun>(v & SWEEP_V_COARSE, v & SWEEP_V_LO, v & SWEEP_V_RESTRICT,
                                         !(v & SWEEP_V_NOGHOST), (v & SWEEP_V_DEV16) ? 1 : (v & SWEEP_V_DEVBF16) ? 2 : 0,
                                         (v & SWEEP_V_TILE) != 0, P, s);
}

template <typename T, typename TC>
int sweep_slots_impl(int v)
{
    return dispatch_kind<T, TC, SlotsRun>(v & SWEEP_V_COARSE, v & SWEEP_V_LO, v & SWEEP_V_RESTRICT, !(v & SWEEP_V_NOGHOST),
                                          (v & SWEEP_V_DEV16) ? 1 : (v & SWEEP_V_DEVBF16) ? 2 : 0);
}

}  // namespace biot

// sweep_chain.cuh -- several smoothing sweeps of one small FP64 level in a single
// launch (the coarsest level of the V-cycle), built on the tile sweep of
// sweep_mom.cuh.
#pragma once
#include "sweep_mom.cuh"

namespace biot {

// Consecutive smoothing sweeps of a small FP64 level in one CTA (the coarsest
// level's 2K sweeps of a V-cycle): the tile covers the whole level, so the
// block barrier between sweeps makes every sweep's global writes -- the moments
// and the bounce-back history -- visible to the next one.  The per-cell code is
// that of k_sweep_tile; only the launches between the sweeps are saved.
template <typename T, typename TC, int KIND>
__global__ void __launch_bounds__(TileShape<SWEEP_CHAIN_MAX, SWEEP_CHAIN_MAX>::NT)
    k_sweep_tile_chain(const SweepArgs<T, TC> a0, int n)
{
    constexpr int TX = SWEEP_CHAIN_MAX, TY = SWEEP_CHAIN_MAX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3][TileShape<TX, TY>::NT / 32];
    __shared__ SweepArgs<T, TC> a;
    if (threadIdx.x == 0) a = a0;
    __syncthreads();
    for (int k = 0; k < n; k++) {
        tile_body<T, TC, TX, TY, KIND, false, false>(a, 0, 0, smem_raw, red);
        __syncthreads();
        if (threadIdx.x == 0) {  // the output is the next sweep's input
            T *out = a.gout;
            a.gout = const_cast<T *>(a.g);
            a.g = out;
            a.zero_init = 0;
            a.hist_valid = 1;
        }
        __syncthreads();
    }
}

// Barrier of all threads of the thread-block cluster, with release / acquire
// ordering of their memory accesses at cluster scope (so one CTA's global
// writes of a sweep are seen by the others in the next).
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The same chain spread over a thread-block cluster: CTA (bx, by) of the
// cluster owns the FP64 tile (TileFor<double>: 8 x 2 cells) at that position
// of the level, and a cluster barrier separates the sweeps.  An 8^2 level then
// runs on four SMs: the sweep of the coarsest level is bound by the FP64
// arithmetic of one SM, which the cluster multiplies.
template <typename T, typename TC, int KIND>
__global__ void __launch_bounds__(TileShape<TileFor<T>::X, TileFor<T>::Y>::NT)
    k_sweep_tile_chain_cluster(const SweepArgs<T, TC> a0, int n)
{
    constexpr int TX = TileFor<T>::X, TY = TileFor<T>::Y;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3][TileShape<TX, TY>::NT / 32];
    SweepArgs<T, TC> a = a0;
    for (int k = 0; k < n; k++) {
        tile_body<T, TC, TX, TY, KIND, false, false>(a, blockIdx.x, blockIdx.y, smem_raw, red);
        cluster_sync_all();  // every CTA's outputs (moments, history) written
        T *out = a.gout;     // the output is the next sweep's input
        a.gout = const_cast<T *>(a.g);
        a.g = out;
        a.zero_init = 0;
        a.hist_valid = 1;
    }
}

template <typename T, typename TC>
cudaError_t launch_sweep_chain_impl(const SweepArgs<T, TC> &a, int n, cudaStream_t s)
{
    if constexpr (sizeof(T) != 8) {
        return cudaErrorInvalidValue;  // only FP64 levels are chained
    } else {
        constexpr int TX = SWEEP_CHAIN_MAX, TY = SWEEP_CHAIN_MAX;
        if (a.nx > TX || a.ny > TY || a.Ft || a.glo || a.mode != SWEEP_SMOOTH || a.resmax || a.gc) return cudaErrorInvalidValue;
        auto run = [&](auto kern, size_t smem) -> cudaError_t {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            kern<<<1, TileShape<TX, TY>::NT, smem, s>>>(a, n);
            return cudaGetLastError();
        };
        // a cluster of the level's FP64 tiles (at most 8 CTAs, the portable cluster size)
        constexpr int CX = TileFor<T>::X, CY = TileFor<T>::Y;
        const int gx = (a.nx + CX - 1) / CX, gy = (a.ny + CY - 1) / CY;
        if (gx * gy > 1 && gx * gy <= 8) {
            auto runc = [&](auto kern, size_t smem) -> cudaError_t {
                cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                if (e != cudaSuccess) return e;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3(gx, gy, 1);
                cfg.blockDim = dim3(TileShape<CX, CY>::NT, 1, 1);
                cfg.dynamicSmemBytes = smem;
                cfg.stream = s;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = gx;
                at[0].val.clusterDim.y = gy;
                at[0].val.clusterDim.z = 1;
                cfg.attrs = at;
                cfg.numAttrs = 1;
                return cudaLaunchKernelEx(&cfg, kern, a, n);
            };
            if (a.ghosts)
                return runc(k_sweep_tile_chain_cluster<T, TC, KIND_COARSE>, tile_smem_bytes<T, CX, CY, KIND_COARSE, false>());
            return runc(k_sweep_tile_chain_cluster<T, TC, KIND_COARSE | KIND_NOGHOST>,
                        tile_smem_bytes<T, CX, CY, KIND_COARSE | KIND_NOGHOST, false>());
        }
        if (a.ghosts) return run(k_sweep_tile_chain<T, TC, KIND_COARSE>, tile_smem_bytes<T, TX, TY, KIND_COARSE, false>());
        return run(k_sweep_tile_chain<T, TC, KIND_COARSE | KIND_NOGHOST>,
                   tile_smem_bytes<T, TX, TY, KIND_COARSE | KIND_NOGHOST, false>());
    }
}

}  // namespace biot

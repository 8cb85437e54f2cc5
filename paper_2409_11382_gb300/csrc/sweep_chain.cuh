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
        if (a.ghosts) return run(k_sweep_tile_chain<T, TC, KIND_COARSE>, tile_smem_bytes<T, TX, TY, KIND_COARSE, false>());
        return run(k_sweep_tile_chain<T, TC, KIND_COARSE | KIND_NOGHOST>,
                   tile_smem_bytes<T, TX, TY, KIND_COARSE | KIND_NOGHOST, false>());
    }
}

}  // namespace biot

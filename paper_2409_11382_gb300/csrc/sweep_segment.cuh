// sweep_segment.cuh -- the sweeps of the small coarse levels of a V-cycle
// (a segment) in one launch: one thread-block cluster per program, the tiles of
// each sweep spread over the cluster's CTAs, a cluster barrier between sweeps.
// The per-cell code is the tile sweep of sweep_mom.cuh; only the launches
// between the sweeps are saved.
#pragma once
#include "sweep_chain.cuh"
#include "sweep_mom.cuh"

namespace biot {

// Block shape of a segment launch: the tile shape of the family's storage type.
template <typename T>
struct SegShape {
    static constexpr int TX = TileFor<T>::X, TY = TileFor<T>::Y, NT = TileShape<TX, TY>::NT;
};

template <typename T, int KIND>
constexpr size_t seg_smem_bytes()
{
    return tile_smem_bytes<T, SegShape<T>::TX, SegShape<T>::TY, KIND, false>();
}

// The tiles of one sweep that fall to CTA `rank` of a cluster of cs CTAs.
template <typename T, typename TC, int KIND>
__device__ __forceinline__ void seg_tiles(const SweepArgs<T, TC> &a, bool rs, int rank, int cs, unsigned char *smem,
                                          double (&red)[3][SegShape<T>::NT / 32])
{
    constexpr int TX = SegShape<T>::TX, TY = SegShape<T>::TY;
    const int gx = (a.nx + TX - 1) / TX, n = gx * ((a.ny + TY - 1) / TY);
    for (int t = rank; t < n; t += cs) {
        if (rs) tile_body<T, TC, TX, TY, KIND, false, true>(a, t % gx, t / gx, smem, red);
        else tile_body<T, TC, TX, TY, KIND, false, false>(a, t % gx, t / gx, smem, red);
        __syncthreads();  // the tile's shared memory is free for the next one
    }
}

// CTA blockIdx.x runs program blockIdx.x / cs as rank blockIdx.x % cs of its
// cluster (the cluster spans cs consecutive CTAs).  Job k+1 reads what every
// CTA of the cluster wrote in job k (iterates, history, restricted residuals):
// the cluster barrier orders those global accesses.
template <typename T, int KIND>
__global__ void __launch_bounds__(SegShape<T>::NT) k_sweep_segment(const __grid_constant__ SegParams P, int cs)
{
    constexpr int NT = SegShape<T>::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[3][NT / 32];
    __shared__ __align__(16) SegLevel cur;  // the current job's arguments
    const int prog = blockIdx.x / cs, rank = blockIdx.x % cs;
    const int l0 = P.lev0[prog];
    for (int j = P.job0[prog]; j < P.job0[prog + 1]; j++) {
        const unsigned w = P.job[j];
        const SegLevel &L = P.lev[l0 + (w & SEGJ_LEVEL)];
        {  // copy the level record, then patch it
            const int *src = reinterpret_cast<const int *>(&L);
            int *dst = reinterpret_cast<int *>(&cur);
            for (int i = threadIdx.x; i < (int)(sizeof(SegLevel) / sizeof(int)); i += NT) dst[i] = src[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if constexpr (sizeof(T) == 8) seg_patch<double, double>(cur.a.dd, L, w);
            else if (L.tkind == 1) seg_patch<float, double>(cur.a.fd, L, w);
            else seg_patch<float, float>(cur.a.ff, L, w);
        }
        __syncthreads();
        const bool rs = (w & SEGJ_RESTRICT) != 0;
        if constexpr (sizeof(T) == 8) {
            seg_tiles<double, double, KIND>(cur.a.dd, rs, rank, cs, smem_raw, red);
        } else {
            if (cur.tkind == 1) seg_tiles<float, double, KIND>(cur.a.fd, rs, rank, cs, smem_raw, red);
            else seg_tiles<float, float, KIND>(cur.a.ff, rs, rank, cs, smem_raw, red);
        }
        cluster_sync_all();  // every CTA's outputs of this sweep written and visible
    }
}

template <typename T, int KIND>
cudaError_t launch_segment_kind(const SegParams &P, int cs, cudaStream_t s)
{
    constexpr size_t smem = seg_smem_bytes<T, KIND>();
    auto kern = k_sweep_segment<T, KIND>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.nprog * cs, 1, 1);
    cfg.blockDim = dim3(SegShape<T>::NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, P, cs);
}

template <typename T>
cudaError_t launch_sweep_segment_impl(const SegParams &P, int cs, cudaStream_t s)
{
    if (P.nprog < 1 || P.nprog > SEG_MAX_PROGS || cs < 1 || cs > SEG_CLUSTER) return cudaErrorInvalidValue;
    if (P.ghosts) return launch_segment_kind<T, KIND_COARSE>(P, cs, s);
    return launch_segment_kind<T, KIND_COARSE | KIND_NOGHOST>(P, cs, s);
}

}  // namespace biot

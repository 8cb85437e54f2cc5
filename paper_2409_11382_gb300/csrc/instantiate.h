// instantiate.h -- explicit specialisations of the launchers for one
// precision; included once by each kernels_*.cu translation unit.
#pragma once
#include "field_kernels.cuh"
#include "sweep_batch.cuh"
#include "sweep_chain.cuh"
#include "sweep_mom.cuh"
#include "sweep_segment.cuh"

#define BIOT_SWEEP_MOM(T, TC)                                                                          \
    template <> cudaError_t biot::launch_sweep_mom<T, TC>(const biot::SweepArgs<T, TC> &a, cudaStream_t s) \
    { return biot::launch_sweep_mom_impl<T, TC>(a, s); }                                               \
    template <> cudaError_t biot::launch_sweep_batch<T, TC>(int v, const biot::BatchParams<T, TC> &P,   \
                                                            cudaStream_t s)                            \
    { return biot::launch_sweep_batch_impl<T, TC>(v, P, s); }                                          \
    template <> int biot::sweep_slots<T, TC>(int v) { return biot::sweep_slots_impl<T, TC>(v); }       \
    template <> int biot::sweep_strip_slots<T, TC>(int v) { return biot::sweep_strip_slots_impl<T, TC>(v); } \
    template <> cudaError_t biot::launch_sweep_chain<T, TC>(const biot::SweepArgs<T, TC> &a, int n,     \
                                                            cudaStream_t s)                            \
    { return biot::launch_sweep_chain_impl<T, TC>(a, n, s); }
#define BIOT_SEGMENT(T)                                                                                \
    template <> cudaError_t biot::launch_sweep_segment<T>(const biot::SegParams &P, int cs, cudaStream_t s) \
    { return biot::launch_sweep_segment_impl<T>(P, cs, s); }
#define BIOT_FIELDS(T)                                                                                 \
    template <> cudaError_t biot::launch_sexp<T>(const biot::SexpArgs<T> &a, cudaStream_t s)             \
    { return biot::launch_sexp_impl<T>(a, s); }                                                        \
    template <> cudaError_t biot::launch_force<T>(const biot::ForceArgs<T> &a, cudaStream_t s)           \
    { return biot::launch_force_impl<T>(a, s); }                                                       \
    template <> cudaError_t biot::launch_readout<T>(const biot::ReadoutArgs<T> &a, cudaStream_t s)       \
    { return biot::launch_readout_impl<T>(a, s); }                                                     \
    template <> cudaError_t biot::launch_init<T>(const biot::InitArgs<T> &a, cudaStream_t s)             \
    { return biot::launch_init_impl<T>(a, s); }                                                        \
    template <> cudaError_t biot::launch_flow_fused<T>(const biot::FlowFusedArgs<T> &a, cudaStream_t s) \
    { return biot::launch_flow_fused_impl<T>(a, s); } \
    template <> cudaError_t biot::launch_flow_fused_batch<T>(const biot::FlowFusedArgs<T> *j,            \
                                                             const biot::SweepItem *it, int n, cudaStream_t s) \
    { return biot::launch_flow_fused_batch_impl<T>(j, it, n, s); }

// Stored-matrix (SELL) Clenshaw sweeps at the launch shape of 1 slice(s) per
// warp iteration and blocks of up to 1024 threads (one of the shapes the
// autotuner chooses from; the kernel is in sweep_b1.cuh). Kept in a
// translation unit of its own so that the shapes compile in parallel.
#include "sweep_b1.cuh"

namespace tbpm {

cudaError_t launch_sell_s1_b1024(const SweepVariant &v, SweepKind kind, bool a_imag, bool has_z,
                           const SweepParams &p, int grid, cudaStream_t s)
{
    if (v.op != OP_SELL || v.block > 1024) return cudaErrorInvalidValue;
    return sell_shape_launch<1, 1024>(v, kind, a_imag, has_z, p, grid, s);
}

int occupancy_sell_s1_b1024(const SweepVariant &v, bool multi, int kind)
{
    if (v.op != OP_SELL || v.block > 1024) return 0;
    return sell_shape_occupancy<1, 1024>(v, multi, kind);
}

}  // namespace tbpm

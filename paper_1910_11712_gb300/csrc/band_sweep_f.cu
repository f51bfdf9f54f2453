// Banded substitution sweeps, complex FP32 instantiation.
#include "band_sweep.cuh"

namespace nep {
template int band_sweeps<float>(const SplitDev&, int, const cx<float>*, const cx<float>*, const int*, int, cx<float>*,
                              const int*, cudaStream_t, int);
template int band_transpose_u<float>(const SplitDev&, int, const cx<float>*, cx<float>*, cudaStream_t);
template int band_sweeps_batch<float>(int, int, int, int, int, const PointDesc*, cudaStream_t);
template void sweep_key<float>(int, int, int, int, int*, int*, int*, int);
}  // namespace nep

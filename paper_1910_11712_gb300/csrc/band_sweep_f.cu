// Banded substitution sweeps, complex FP32 instantiation.
#include "band_sweep.cuh"

namespace nep {
template int band_sweeps<float>(const SplitDev&, int, const cx<float>*, const cx<float>*, const int*, int, cx<float>*,
                              const int*, cudaStream_t);
template int band_transpose_u<float>(const SplitDev&, int, const cx<float>*, cx<float>*, cudaStream_t);
}  // namespace nep

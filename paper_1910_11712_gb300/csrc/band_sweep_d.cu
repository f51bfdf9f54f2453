// Banded substitution sweeps, complex FP64 instantiation.
#include "band_sweep.cuh"

namespace nep {
template int band_sweeps<double>(const SplitDev&, int, const cx<double>*, const cx<double>*, const int*, int, cx<double>*,
                              const int*, cudaStream_t, int);
template int band_transpose_u<double>(const SplitDev&, int, const cx<double>*, cx<double>*, cudaStream_t);
template int band_sweeps_batch<double>(int, int, int, int, int, const PointDesc*, cudaStream_t);
template void sweep_key<double>(int, int, int, int, int*, int*, int*, int);
}  // namespace nep

// float instantiation of the adjoint pair kernel: the table (mixed-precision) path.
#include "pair_adj.cuh"

template cudaError_t sg_pair_adjoint<float>(const AdjArgs<float>&, int, bool, cudaStream_t);

// double instantiation of the adjoint pair kernel: the recursion (FP64) path.
#include "pair_adj.cuh"

template cudaError_t sg_pair_adjoint<double>(const AdjArgs<double>&, int, bool, cudaStream_t);

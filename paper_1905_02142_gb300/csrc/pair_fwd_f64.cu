// double instantiation of the forward pair kernel: the recursion (FP64) path.
#include "pair_fwd.cuh"

template cudaError_t sg_pair_forward<double>(const FwdArgs<double>&, int, bool, cudaStream_t);

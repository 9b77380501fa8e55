// float instantiation of the forward pair kernel: the table (mixed-precision) path.
#include "pair_fwd.cuh"

template cudaError_t sg_pair_forward<float>(const FwdArgs<float>&, int, bool, cudaStream_t);

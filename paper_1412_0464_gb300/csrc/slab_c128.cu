// Complex128 instantiation of the slab factorisation and slab solves.
#include "slab.cuh"

namespace hz {
template void factor_level<double>(hz_handle*, Level&, cudaStream_t);
template void subdom_solve<double>(hz_handle*, Level&, int, const c128*, int, int, int, int, bool,
                                   const c128*, bool, c128*, bool, const c128*, bool, c128*, c128*,
                                   int, cudaStream_t);
template void slab_solve_raw<double>(hz_handle*, Level&, int, const c128*, c128*, int, cudaStream_t);
template void slab_solve_raw_scratch<double>(hz_handle*, Level&, int, const c128*, c128*, int,
                                             cudaStream_t, c128*, c128*, c128*);
}  // namespace hz

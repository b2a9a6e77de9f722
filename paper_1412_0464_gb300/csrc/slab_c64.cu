// Complex64 instantiation of the slab factorisation and slab solves.
#include "slab.cuh"

namespace hz {
template void factor_level<float>(hz_handle*, Level&, cudaStream_t);
template void subdom_solve<float>(hz_handle*, Level&, int, const c64*, int, int, int, int, bool,
                                  const c64*, bool, c64*, bool, const c64*, bool, c64*, c64*, int,
                                  cudaStream_t);
template void slab_solve_raw<float>(hz_handle*, Level&, int, const c64*, c64*, int, cudaStream_t);
template void slab_solve_raw_scratch<float>(hz_handle*, Level&, int, const c64*, c64*, int,
                                            cudaStream_t, c64*, c64*, c64*);
}  // namespace hz

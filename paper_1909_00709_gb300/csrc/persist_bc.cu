// Persistent launches of grids with periodic boundaries: the kernels of persist.cuh
// instantiated with tile policies for that rule (a translation unit of its own, so the
// rules' kernels compile in parallel).
#include <cstring>

#include "persist.cuh"

namespace abft {

bool persistent_fits_periodic(const GridDev& g, bool prot) { return persistent_fits_cl<ABFT_BC_PERIODIC>(g, prot); }

cudaError_t launch_persistent_periodic(const Launch& L, const PersistArgs& a, bool prot, int* blocks) {
  return launch_persistent_cl<ABFT_BC_PERIODIC>(L, a, prot, blocks);
}

cudaError_t launch_offline_periodic(const Launch& L, const PersistArgs& a, int* blocks) {
  return launch_offline_cl<ABFT_BC_PERIODIC>(L, a, blocks);
}

bool persistent_offline_fits_periodic(const GridDev& g) { return offline_fits_cl<ABFT_BC_PERIODIC>(g); }

}  // namespace abft

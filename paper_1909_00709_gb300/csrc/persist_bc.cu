// Persistent launches of grids with a periodic or empty boundary: the kernels of
// persist.cuh instantiated with tile policies that read the rule from the grid
// descriptor (a translation unit of its own, so the two sets compile in parallel).
#include <cstring>

#include "persist.cuh"

namespace abft {

bool persistent_fits_generic(const GridDev& g, bool prot) { return persistent_fits_cl<false>(g, prot); }

cudaError_t launch_persistent_generic(const Launch& L, const PersistArgs& a, bool prot, int* blocks) {
  return launch_persistent_cl<false>(L, a, prot, blocks);
}

cudaError_t launch_offline_generic(const Launch& L, const PersistArgs& a, int* blocks) {
  return launch_offline_cl<false>(L, a, blocks);
}

bool persistent_offline_fits_generic(const GridDev& g) { return offline_fits_cl<false>(g); }

}  // namespace abft

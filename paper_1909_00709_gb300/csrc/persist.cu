// Persistent launches of grids with the clamped boundary (the default) and the public
// entry points; grids with other boundary rules go to persist_bc.cu (periodic) and
// persist_zero.cu (empty).
#include <cstring>

#include "persist.cuh"

namespace abft {

bool persistent_fits(const GridDev& g, bool prot) {
  return g.bc == ABFT_BC_PERIODIC ? persistent_fits_periodic(g, prot)
         : g.bc == ABFT_BC_ZERO   ? persistent_fits_zero(g, prot)
                                  : persistent_fits_cl<ABFT_BC_CLAMP>(g, prot);
}

cudaError_t launch_persistent(const Launch& L, const GridDev& g, const CUtensorMap tm_u[3], const CUtensorMap& tm_c,
                              const CUtensorMap tm_p[4], long long step0, int n_steps, int first_in, int p, int q,
                              bool prot, int* blocks) {
  PersistArgs a;
  for (int k = 0; k < 3; ++k) a.tm_u[k] = tm_u[k];
  for (int k = 0; k < 4; ++k) a.tm_p[k] = tm_p[k];
  a.tm_c = tm_c;
  a.g = g;
  a.step0 = step0;
  a.n_steps = n_steps;
  a.first_in = first_in;
  a.p = p;
  a.q = q;
  return g.bc == ABFT_BC_PERIODIC ? launch_persistent_periodic(L, a, prot, blocks)
         : g.bc == ABFT_BC_ZERO   ? launch_persistent_zero(L, a, prot, blocks)
                                  : launch_persistent_cl<ABFT_BC_CLAMP>(L, a, prot, blocks);
}

cudaError_t launch_persistent_offline(const Launch& L, const GridDev& g, const CUtensorMap tm_u[3],
                                      const CUtensorMap& tm_c, long long step0, int n_steps, int delta, int ck,
                                      int* blocks) {
  PersistArgs a;
  memset(&a, 0, sizeof a);
  for (int k = 0; k < 3; ++k) a.tm_u[k] = tm_u[k];
  a.tm_c = tm_c;
  a.g = g;
  a.step0 = step0;
  a.n_steps = n_steps;
  a.first_in = ck;
  a.delta = delta;
  return g.bc == ABFT_BC_PERIODIC ? launch_offline_periodic(L, a, blocks)
         : g.bc == ABFT_BC_ZERO   ? launch_offline_zero(L, a, blocks)
                                  : launch_offline_cl<ABFT_BC_CLAMP>(L, a, blocks);
}

bool persistent_offline_fits(const GridDev& g) {
  return g.bc == ABFT_BC_PERIODIC ? persistent_offline_fits_periodic(g)
         : g.bc == ABFT_BC_ZERO   ? persistent_offline_fits_zero(g)
                                  : offline_fits_cl<ABFT_BC_CLAMP>(g);
}

}  // namespace abft

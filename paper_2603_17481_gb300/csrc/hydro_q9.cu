// hydro_q9.cu -- instantiation of the hydrodynamic kernel for the D2Q9 lattice (one translation
// unit per lattice so that the three compile in parallel).
#include "hydro_impl.cuh"

namespace lbm {

cudaError_t launch_hydro_q9(int store, int mode, const KParams &P, const void *src, void *dst,
                             const int32_t *phi, const float4 *frep, float *u, float *pstar, cudaStream_t s) {
  return launch_hydro_lattice<D2Q9>(store, mode, P, src, dst, phi, frep, u, pstar, s);
}

}  // namespace lbm

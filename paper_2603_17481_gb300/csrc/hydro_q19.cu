// hydro_q19.cu -- instantiation of the hydrodynamic kernel for the D3Q19 lattice (one translation
// unit per lattice so that the three compile in parallel).
#include "hydro_impl.cuh"

namespace lbm {

cudaError_t launch_hydro_q19(int store, int mode, const KParams &P, const void *src, void *dst,
                             const int32_t *phi, const float4 *frep, float *u, float *pstar, cudaStream_t s) {
  return launch_hydro_lattice<D3Q19>(store, mode, P, src, dst, phi, frep, u, pstar, s);
}

cudaError_t launch_split_q19(int part, int store, const KParams &P, const void *src, void *dst,
                             const int32_t *phi, const float4 *frep, float *u, const TileList &listed, int blocks,
                             cudaStream_t s) {
  return launch_split_lattice<D3Q19>(part, store, P, src, dst, phi, frep, u, listed, blocks, s);
}

}  // namespace lbm

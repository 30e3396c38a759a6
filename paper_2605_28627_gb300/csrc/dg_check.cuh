// Bounds checks of the indirect gathers (debug builds).
//
// Every index a kernel reads from a connectivity table -- a neighbour element
// from the neighbour map, a face id from the element-face codes, the two
// elements of a face descriptor, a member from an ensemble tile -- passes
// through dg_idx.  In builds with -DDG_BOUNDS_CHECK (build(checked=True)) an
// index outside [0, bound) is recorded in this translation unit's error word
// (the first one only: a flag bit, the site number and the index) and replaced
// by 0, so the access that follows stays inside its array and nothing faults;
// the entry points synchronise after their launches and report a recorded
// error as DG_ECUDA.  In normal builds dg_idx returns its argument.  The flip
// codes and the face-node map need no check: every code maps in-range face
// nodes to in-range face nodes.
#pragma once

#include <cuda_runtime.h>

namespace dg {

// Check sites (the reported site number).
enum BoundsSite {
  kSiteLiftNbr = 1,      // lifting: neighbour element of a face point
  kSiteFaceElems = 2,    // face flux: the two elements of a face
  kSiteVolFace = 3,      // volume: face id of an element face (surface integral, prefetch)
  kSiteGaussLift = 4,    // Gauss nodes: lifting neighbour / face id
  kSiteGaussFace = 5,    // Gauss nodes: face flux elements, face geometry
  kSiteGaussVol = 6,     // Gauss nodes: volume face id
  kSiteGeomFace = 7,     // face geometry: master element
  kSiteAdjFace = 8,      // adjoint: face elements, face ids, neighbours
  kSiteEnsMember = 9,    // ensemble: member of a tile
  kSiteFvNbr = 10,       // FV sub-cells: neighbour element across a face
  kSiteFvFace = 11,      // FV sub-cells: face elements, face id of an element face
  kSiteMortar = 12       // mortars: the elements and face slots of a mortar
};

#ifdef DG_BOUNDS_CHECK
static __device__ unsigned long long dg_bounds_word;   // one per translation unit

__device__ __forceinline__ int dg_idx(long v, long bound, int site) {
  if (v >= 0 && v < bound) return (int)v;
  const unsigned long long w =
      (1ull << 63) | ((unsigned long long)(site & 0x7fff) << 48) | ((unsigned long long)v & 0xffffffffffffull);
  atomicCAS(&dg_bounds_word, 0ull, w);
  return 0;
}

// Host reader of this translation unit's word: returns it and clears it.
#define DG_BOUNDS_READER(name)                                            \
  unsigned long long name() {                                             \
    unsigned long long w = 0, z = 0;                                      \
    if (cudaMemcpyFromSymbol(&w, dg_bounds_word, sizeof w) != cudaSuccess) \
      return 0;                                                           \
    cudaMemcpyToSymbol(dg_bounds_word, &z, sizeof z);                     \
    return w;                                                             \
  }
#else
__device__ __forceinline__ int dg_idx(long v, long, int) { return (int)v; }
#define DG_BOUNDS_READER(name) \
  unsigned long long name() { return 0; }
#endif

}  // namespace dg

// batch_table.cuh -- argument sets of one simulation's step, as the kernels
// read them: PushArgs for the tiled particle step (a kernel parameter for one
// simulation or a group of batch members, in param space), and the table
// entry of a batch member (BatchMember, BatchMaps), written by the host once
// per membership and step parity.
#pragma once
#include <cuda.h>

#include "common.cuh"

namespace mithra {

template <typename T, typename U>
struct PushArgs {
  PicP<T> p;
  StepState* st;
  const V4<T>* pn;  // psi^{n+1}
  const V4<T>* D;   // increment
  V4<T>* src;
  Parts<T, U> P;      // the particles, at the positions perm gives
  Parts<T, U> O;      // receives them in slot order (the other buffer)
  const int* perm;    // slot of the tile order -> position in P
  const int* offset;
  const int* tiles;
  int* count;
  int* key;
  int* rank;
  long long* lost_ctr;
  long long np;
  // source-tile flags (StencilP::dirty): two arrays of dirty_words words,
  // the one of parity cur read by this step's potential update (cleared
  // here), the other marked for the next
  unsigned char* dirty;
  int dirty_words;
  int cur;
};

template <typename T, typename U>
struct BatchMember {
  StencilP<T> sp;
  PicP<T> pp;  // pp.plo: lo parts of the level E and B come from
  V4<T>* P0;   // psi^n
  V4<T>* P1;   // receives psi^{n+1}
  LoV4* L0;
  LoV4* L1;
  V4<T>* D;
  V4<T>* S;
  Parts<T, U> A, B;  // particles in use, and the buffer the particle step writes
  int* perm;         // slot of the tile order -> position in A (the re-sort's output)
  int* offset;
  int* tiles;
  int* count;
  int* key;
  int* rank;
  int4* scan_part;
  StepState* st;
  double* power_acc;    // record base minus the first recorded step
  long long power_end;  // first + capacity (0: no recording)
  double g0, b0;        // frame of the power transformation
  long long np;
  int lz;
  int power_plane;
  int nkeys;
  int scan_nb;
  int sparse_below;
  int fused_mur;  // first-order Mur at the x faces inside the z-marching loop
  unsigned char* dirty;  // source-tile flags, as in PushArgs
  int dirty_words;
  int cur;
};

// Tensor maps of a member's particle step, collected on the host (the
// kernels take them in their parameter space).
struct BatchMaps {
  CUtensorMap box;    // psi^{n+1}, 11^3 boxes
  CUtensorMap box_d;  // increment, 11^3 boxes
};

}  // namespace mithra

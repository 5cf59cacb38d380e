// tm_batch.cuh -- device structures of the batched solver (tm_batch.cu) shared with its
// K-systems-per-thread hopping kernel (tm_batch_group.cu).
#pragma once

#include <algorithm>

#include "tm_dslash.cuh"

namespace tmq {

// Per-system descriptor (device memory).
struct BatchSys {
  Geom g;
  const char* links;   // sloppy gauge copy of the system's lattice
  EpiCoef coef[4];     // epilogues of K1..K4 (this system's mu)
  void* vec[5];        // 0 p, 1 T, 2 W (sloppy storage), 3 r, 4 x increment (FP32)
  CGState* st;
  double* partials;    // reduction partials of this system (nblocks entries)
  unsigned* counters;  // [0] reductions, [1] update kernel
  int nblocks;         // blocks of the hopping launch this table serves (hop_spb(TPS) sites each)
  int nblocks_upd;     // update-kernel blocks
  double* result;      // the FP64 service's ||b' - A X||^2 (reductions of kind FIN_STORE)
};

struct BatchGlobal {
  int unfinished;    // systems not yet done for good
  int loops;         // iterations executed (bodies of the graph loop)
  int loop_cap;      // hard bound on loops
  unsigned counter;  // update-kernel blocks arrived
  int nsys;          // systems in the batch
  int services;      // executions of the FP64 service
  double delta2;     // reliable-update trigger of a resumed system
  double grow2;      // divergence guard of a resumed system
};

// A work list: the live systems of the batch, compacted lattice by lattice and rebuilt inside the
// graph whenever the set of running systems changes.  Virtual block v of a launch belongs to the
// lattice li with start[li] <= v < start[li + 1]; there it is block (v - start[li]) / count[li] of
// system items[base[li] + (v - start[li]) % count[li]], so the systems of one lattice take turns
// block by block, read each link at about the same time and share it through L2.  Launches hold
// as many blocks as the GPU keeps resident and walk the list with a stride: the blocks of stopped
// and finished systems cost nothing.
struct Plan {
  int nlat;
  const int* base;    // [nlat] first candidate (and item slot) of lattice li
  const int* ncand;   // [nlat] candidates on lattice li
  const int* blocks;  // [nlat] blocks per system on lattice li (of the launch the list serves)
  int* start;         // [nlat + 1] first virtual block of lattice li; start[nlat] = the total
  int* count;         // [nlat] live systems on lattice li
  int* items;         // the live systems, lattice li's from base[li]
};

// Up to 4 systems of one lattice whose hopping terms one thread computes together (the
// K-systems-per-thread kernel): their indices in the system table, the first one's geometry and
// links serving all.
struct BatchGroup {
  int n;
  int sys[4];
};

// The work lists of a batched solve: the running systems' hopping and update blocks, and the
// FP64 service's for the systems that stopped (candidates: the positions in `order`); and the
// running groups' blocks for the K-systems-per-thread kernel (candidates: the group ids).
struct Plans {
  Plan hop, upd, shop, supd, ghop;
  const int* order;           // [nsys] system ids, lattice by lattice
  CGState* states;            // [nsys] the systems' CG states
  const BatchGroup* groups;   // [ngroups] the groups, lattice by lattice
};

__device__ __forceinline__ int2 plan_item(const Plan& P, int v) {
  int li = 0;
  while (li + 1 < P.nlat && v >= P.start[li + 1]) ++li;
  const int w = v - P.start[li];
  const int c = P.count[li];
  return make_int2(P.items[P.base[li] + w % c], w / c);
}

// The hopping launch of K = 2 or 4 systems per thread over the groups of a work list
// (tm_batch_group.cu): FP32 or FP16 storage, HOP_NT sites per block.
tm_status launch_hop_group(int prec, int nreal, int K, const BatchSys* d_sys, const BatchGroup* d_grp,
                           const CGState* d_st, const Plan& plan, int cap, int in_sel, int y_sel, int out_sel, int kk,
                           int parity, int mode, bool has_y, cudaStream_t s);

// Blocks of a launch: as many as the GPU keeps resident (at most `cap`, the blocks of a full list).
template <class Kern>
inline int resident_grid(Kern kern, int threads, int cap) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, 0);
  return std::max(1, std::min(cap, std::max(1, per) * std::max(1, nsm)));
}

}  // namespace tmq

// Launch entry points shared between the host API and the kernel translation
// units. Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace cglbm {

// block size of the phase-by-phase kernels: 128 threads, small enough for a
// block to run beside the bulk kernel's CTAs on an SM
constexpr int kBoxThreads = 128;

// The fused kernels split each tile column's nz planes into
// ceil(nz / zchunk) chunks of near-equal length (chunk k is
// [k nz / n, (k + 1) nz / n)), so that the chunk count, and with it the number
// of waves of CTAs, can be chosen freely without a short last chunk.
__host__ __device__ inline int z_chunks(int nz, int zchunk) { return (nz + zchunk - 1) / zchunk; }
__host__ __device__ inline int z_chunk_begin(int nz, int n, int k) { return (int)((long long)k * nz / n); }

// Phase-by-phase step over region R (all sites, or the nozzle box):
//   0. per-column nozzle flags over R grown by four rings (nozzle runs)
//   1. stream + densities on R grown by two rings, ledger of R
//   2. created nodes on R grown by one ring
//   3. fictitious wall densities and ghost planes on R grown by one ring
//   4. collision on R
// Returns the number of kernels launched.
// S is the stored population type (see Stored).
template <class VS, typename real, typename S>
int launch_plain(const StepArgs<real>& p, const Region& R, const Region& R1, const Region& R2, cudaStream_t st);

// Fused bulk step over every site outside p.box (D3Q19, substrate + open top).
template <typename real, typename S>
int launch_fused(const StepArgs<real>& p, int zchunk, cudaStream_t st);

// Persistent fused bulk step over many lattices in one launch: grid CTAs take
// the work list items (lattice index, x0 | y0 << 16, za, zb: one tile column
// of planes [za, zb)) in order through the counter *queue (zero at launch),
// reading each lattice's StepArgs from args (device). All lattices share the
// kernel configuration (unit flag). With occupancy != NULL nothing is
// launched and the resident CTAs per SM of that configuration are returned
// there.
template <typename real, typename S>
int launch_fused_batch(const StepArgs<real>* args, const int4* items, int n_items, int* queue, int grid, int unit,
                       cudaStream_t st, int* occupancy);
// tile height (sites in y) of the batched fused kernel's 32-wide column tiles
constexpr int kFusedTileH = 8;
// resident CTAs per SM of the single-lattice fused kernel (32 x 8 tiles):
// three in FP32 arithmetic, one in FP64
inline int fused_ctas_per_sm(bool fp64) { return fp64 ? 1 : 3; }

// Batched phase-by-phase step of the nozzle boxes of many lattices: one
// launch per phase over all lattices (blockIdx.z), each lattice's StepArgs
// and regions read from the device table t; gx, gy: the largest grid of a
// lattice's grown box (columns, planes).
template <typename real>
struct BoxArgs {
    StepArgs<real> p;
    Region R, R1, R2, R1g, Rg;  // Rg: the columns of the nozzle flags (R2 and two more rings)
};
template <class VS, typename real, typename S>
int launch_plain_batch(const BoxArgs<real>* t, int n, unsigned gx, unsigned gy, int unit, cudaStream_t st);

// Equilibrium initialisation from fields staged in p.fields (rho_ink, rho_amb,
// ux, uy, uz planes; u optional) or, when staged == 0, from the print-setup
// default (ink inside the nozzle above the gap, ambient elsewhere, at rest).
template <class VS, typename real, typename S>
int launch_init(const StepArgs<real>& p, int staged, int have_u, cudaStream_t st);

// Rebuild (plain storage only) the previous step's densities (every fluid node of the step-(n-1)
// geometry) and the physical velocity of the last two planes from the
// post-collision populations p.fin: collision conserves each component's
// mass, and its momentum is rho u + F (exact difference method).
template <class VS, typename real>
int launch_prev_from_f(const StepArgs<real>& p, real* rho_prev, real* u_prev, cudaStream_t st);

}  // namespace cglbm

// Launch entry points shared between the host API and the kernel translation
// units. Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace cglbm {

// Phase-by-phase step over region R (all sites, or the nozzle box):
//   1. stream + densities on R grown by two rings, ledger of R
//   2. created nodes on R grown by one ring
//   3. fictitious wall densities and ghost planes on R grown by one ring
//   4. collision on R
// Returns the number of kernels launched.
// S is the stored population type (see Stored).
template <class VS, typename real, typename S>
int launch_plain(const StepArgs<real>& p, const Region& R, const Region& R1, const Region& R2, cudaStream_t st);

// Fused bulk step over every site outside p.box (D3Q19, substrate + open top).
// variant selects a tile/staging configuration (0 = default).
template <typename real, typename S>
int launch_fused(const StepArgs<real>& p, int zchunk, cudaStream_t st, int variant);

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

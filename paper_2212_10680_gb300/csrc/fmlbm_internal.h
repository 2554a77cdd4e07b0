// Host helpers shared between the single-lattice and the batch/serve parts of the C ABI.
#pragma once

#include <string>

#include "fmlbm.h"
#include "fmlbm_kernels.cuh"

// Appendix C constants of a mixture (a_i, b_i, alpha_i(T), (a alpha)_ij, kappa_ij);
// false with a reason when the mixture is invalid.
bool fmlbm_internal_mixture_constants(const fmlbm_mixture& m, fmlbm::MixConst* mc, std::string* why);
// Validity of a lattice description for n components.
bool fmlbm_internal_lattice_ok(const fmlbm_lattice& L, int nc, std::string* why);
// A device (or managed) allocation on `device`, aligned to `align` bytes, with at least
// `bytes` from p to the end of the allocation that contains it.
bool fmlbm_internal_usable_device_pointer(const void* p, size_t bytes, int device, size_t align = 16);
// Restricts the domain check of a handle's steps to rows [y0, y1) (y1 = 0: all rows): a slab
// of a decomposed lattice checks its own rows, not its ghost rows.
void fmlbm_internal_set_check_rows(fmlbm_handle* h, int y0, int y1);

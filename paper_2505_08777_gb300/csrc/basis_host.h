// Host-side Zernike monomial tables (fp64); see basis_host.cpp.
#pragma once

#include <vector>

#include "mono.h"

namespace ash {

// Noll index j (>= 1) -> radial order n and signed azimuthal order m
// (m > 0 cosine, m < 0 sine). Returns false for an invalid index.
bool noll_to_nm(int j, int* n, int* m);

// Appends the nonzero monomial terms of the unnormalised Zernike Z_n^m.
bool zernike_monomials(int n, int m, std::vector<MonoTerm>* out);

}  // namespace ash

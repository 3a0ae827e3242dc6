// Monomial term of a basis polynomial (shared by the host table builder and
// the basis kernel).
#pragma once

namespace ash {

// coef * x^px * y^py
struct MonoTerm {
  double coef;
  int px, py;
};

}  // namespace ash

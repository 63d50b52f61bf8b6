// sl1m_sincos_poly.h -- generated by gen_sincos_poly.py (Chebyshev interpolation,
// degree 4 in z = f^2 on [0, 1/4]); do not edit by hand.
//   sqrt(2) sin(pi f) = f * P(z),  sqrt(2) cos(pi f) = Q(z),  f in [-1/2, 1/2]
#pragma once

namespace sl1m {
constexpr float SCP0 = 4.442883014678955f;
constexpr float SCP1 = -7.308245658874512f;
constexpr float SCP2 = 3.606353998184204f;
constexpr float SCP3 = -0.8461104035377502f;
constexpr float SCP4 = 0.10982204228639603f;
constexpr float SCQ0 = 1.4142135381698608f;
constexpr float SCQ1 = -6.978850841522217f;
constexpr float SCQ2 = 5.73945951461792f;
constexpr float SCQ3 = -1.8835527896881104f;
constexpr float SCQ4 = 0.3106778562068939f;

}  // namespace sl1m

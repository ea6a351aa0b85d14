// quantile_f32.h -- written by gen_quantile_f32.py (40-digit mpmath); do not edit.
#pragma once

namespace lsmc {

// Phi^-1(u) = x P(w - 2.5) (w < 5) or x Q(sqrt(w) - 3) (w >= 5), x = 2u - 1,
// w = -log(4 u (1 - u)); P(t) = sum kQfP<k> t^k, Q(s) = sum kQfQ<k> s^k.
constexpr float kQfNegLn2 = -6.931471825e-01f;  // -ln 2
constexpr float kQfShift = -3.886294365e+00f;   // -2 ln 2 - 2.5
constexpr float kQfSplit = 2.5f;             // w = 5
constexpr float kQfP0 = 2.123313665e+00f;
constexpr float kQfP1 = 3.488026857e-01f;
constexpr float kQfP2 = -5.908129737e-03f;
constexpr float kQfP3 = -1.773041789e-03f;
constexpr float kQfP4 = 3.091151011e-04f;
constexpr float kQfP5 = -6.207880233e-06f;
constexpr float kQfP6 = -4.981194706e-06f;
constexpr float kQfP7 = 4.851791005e-07f;
constexpr float kQfP8 = 3.958320960e-08f;
constexpr float kQfQ0 = 4.006434441e+00f;
constexpr float kQfQ1 = 1.416581154e+00f;
constexpr float kQfQ2 = 1.335394569e-02f;
constexpr float kQfQ3 = -1.077862084e-02f;
constexpr float kQfQ4 = 8.076463826e-03f;
constexpr float kQfQ5 = -5.204700399e-03f;
constexpr float kQfQ6 = 2.004438778e-03f;
constexpr float kQfQ7 = 1.564540871e-04f;
constexpr float kQfQ8 = -3.547589877e-04f;

}  // namespace lsmc

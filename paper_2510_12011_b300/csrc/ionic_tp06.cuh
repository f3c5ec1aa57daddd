// ten Tusscher-Panfilov 2006 human ventricular model: device kernel and resting state.
//
// The paper's volume-mesh runs use this model (Section 2.2, Section 3.3) without printing it;
// the equations follow the model's own publication (ten Tusscher & Panfilov, Am J Physiol
// Heart Circ Physiol 291:H1088, 2006) in its rapid-buffering differential form.  Units: mV, ms,
// mM, currents in pA/pF (multiplied by Cm in uF/mm^2 they are uA/mm^2).
//
// State layout: SoA, state[j * n + i] for node i, j =
//   0 Ki  1 Nai  2 Cai  3 CaSR  4 CaSS  5 Rbar  6 xr1  7 xr2  8 xs  9 m  10 h  11 j
//   12 d  13 f  14 f2  15 fCass  16 s  17 r
// Step (operator splitting of Eq. 2 with Rush-Larsen gates): all rates at (V^k, u^k); gates by
// u_inf + (u - u_inf) exp(-dt/tau); concentrations and Rbar by forward Euler; then
// I_ion(V^k, u^{k+1}).  The stimulus does not enter Ki (it is applied through the PDE source).
#pragma once

#include <cmath>
#include "kernels.cuh"

namespace tc {

constexpr int kTP06States = 18;

namespace tp06 {
constexpr double kR = 8314.472, kT = 310.0, kF = 96485.3415;
constexpr double kRTF = kR * kT / kF;
constexpr double kCap = 0.185, kVc = 0.016404, kVsr = 0.001094, kVss = 0.00005468;
constexpr double kKo = 5.4, kNao = 140.0, kCao = 2.0;
constexpr double kGNa = 14.838, kGK1 = 5.405, kGKr = 0.153, kGpK = 0.0146, kGpCa = 0.1238;
constexpr double kGbNa = 0.00029, kGbCa = 0.000592, kGCaL = 3.98e-5;
constexpr double kPKNa = 0.03, kKpCa = 0.0005, kPNaK = 2.724, kKmK = 1.0, kKmNa = 40.0;
constexpr double kKNaCa = 1000.0, kKmNai = 87.5, kKmCa = 1.38, kKsat = 0.1, kGam = 0.35;
constexpr double kAlphaNaCa = 2.5;
constexpr double kVmaxUp = 0.006375, kKup = 0.00025, kVrel = 0.102, kVleak = 0.00036;
constexpr double kVxfer = 0.0038, kK1p = 0.15, kK2p = 0.045, kK3 = 0.06, kK4 = 0.005;
constexpr double kEC = 1.5, kMaxSR = 2.5, kMinSR = 1.0;
constexpr double kBufc = 0.2, kKbufc = 0.001, kBufsr = 10.0, kKbufsr = 0.3, kBufss = 0.4;
constexpr double kKbufss = 0.00025;
constexpr double kRestV = -85.23;
// natural logarithms of the constant concentrations of the Nernst potentials (Ko, Nao,
// Ko + pKNa Nao, Cao), written out so that no logarithm of a constant is left to run time
constexpr double kLnKo = 1.6863989535702288, kLnNao = 4.941642422609304;
constexpr double kLnKsNa = 2.2617630984737906, kLnCao = 0.6931471805599453;
// exp(b) for the offsets b of gate exponents exp(a V + b) that share a slope a with another
// (then exp(a V + b) = exp(a V) exp(b): one exponential per slope)
constexpr double kE7 = 1096.6331584284585, kE4 = 54.598150033144236, kEm4 = 0.01831563888873418;
constexpr double kE5p6 = 270.42640742615254, kE1 = 2.718281828459045, kEm4p5 = 0.011108996538242306;
constexpr double kE1p3 = 3.6692966676192444, kE2p5 = 12.182493960703473, kEm3p2 = 0.04076220397836621;
constexpr double kE5o6 = 2.300975890892825, kE20o6 = 28.03162489452614, kE20o7 = 17.41170806332765;
constexpr double kE5 = 148.4131591025766, kEm3 = 0.049787068367863944;
// the same device for slopes whose exponential is the reciprocal (or the square of one) of a
// shared one: exp(-12), exp(-26/7), exp(-35/15), exp(-8/7.5), exp(3), and exp(-30 F/RT) (the
// GHK exponential exp(2 (V - 15) F/RT) = exp(-30 F/RT) / exp(-V F/RT)^2)
constexpr double kEm12 = 6.14421235332821e-06, kEm26o7 = 0.0243728440732796;
constexpr double kEm35o15 = 0.09697196786440507, kEm8o7p5 = 0.34415378686541237;
constexpr double kE3 = 20.085536923187668, kGhkK = 0.32529698149690256;
}  // namespace tp06

inline void tp06_rest_state(int /*cell*/, double* u, double* v0) {
  const double r[kTP06States] = {136.89, 8.604,   0.000126, 3.64,   0.00036, 0.9073,
                                 0.00621, 0.4712, 0.0095,   0.00172, 0.7444, 0.7045,
                                 3.373e-5, 0.7888, 0.9755,  0.9953, 0.999998, 2.42e-8};
  for (int j = 0; j < kTP06States; ++j) u[j] = r[j];
  *v0 = tp06::kRestV;
}

// FP64 exponential, table-driven (Tang, ACM TOMS 15(2), 1989): x = (2048 m + j) ln2/2048 + r
// with |r| <= ln2/4096, exp(x) = 2^m * 2^(j/2048) * exp(r), exp(r) - 1 by r + c2 r^2 + r^3/6
// with c2 the equioscillating quadratic coefficient (maximum error 5.9e-18; math_tables.py
// derives it).  ln2/2048 is split into hi + lo so that r is exact to FP64 rounding; 2^(j/2048) is
// a hi + lo pair (th, tl) from a per-block shared-memory table (32 KB) and the result is
// th + (th p + tl), the term tl p (below 2e-20 relative) left out, so the result is within about
// half an ulp; 2^m is added to the exponent field.  Nine FP64 instructions; the range test runs
// on the integer pipe (|x| >= 512, inf and NaN go to the library exp).
constexpr double kExpC2 = 0x1.000000087db8cp-1;
// base 2: 2^r - 1 = r (a1 + r (a2 + r a3)) on |r| <= 2^-12 (the polynomial above in s = r ln 2)
constexpr double kExp2A1 = 0x1.62e42fefa39efp-1, kExp2A2 = 0x1.ebfbe0087dd4fp-3, kExp2A3 = 0x1.c6b08d704a0c0p-5;
constexpr double kLog2e = 0x1.71547652b82fep+0;   // 1 / ln 2
#include "exp2_table.inc"
// Natural logarithm, table method (Tang 1990): for positive normal x = 2^e m, m in [1, 2), take
// F = 1 + j/128 with j the top seven fraction bits of m and c = fl(1/F); then r = m c - 1 (one
// FMA, exact before its final rounding, 0 <= r < 2^-7) and ln x = e ln2 - ln c + log1p(r), with
// -ln c from a hi + lo table (of the rounded reciprocal itself, so the rounding of c costs
// nothing) and log1p(r) by its Taylor polynomial to r^8 (truncation < 2^-63).  ln2 is split into
// hi (43 bits, so that e ln2_hi is exact) + lo.  Other x (zero, negative, subnormal, inf, NaN)
// go to the library log.  The tables (and the 2^(j/2048) pairs above) are regenerated by
// math_tables.py beside this file.
// kLogInv[j] = fl(1/(1 + j/128)); kLogHi[j] + kLogLo[j] = -ln(kLogInv[j])
static __constant__ double kLogInv[128] = {
    0x1.0000000000000p+0, 0x1.fc07f01fc07f0p-1, 0x1.f81f81f81f820p-1,
    0x1.f44659e4a4271p-1, 0x1.f07c1f07c1f08p-1, 0x1.ecc07b301ecc0p-1,
    0x1.e9131abf0b767p-1, 0x1.e573ac901e574p-1, 0x1.e1e1e1e1e1e1ep-1,
    0x1.de5d6e3f8868ap-1, 0x1.dae6076b981dbp-1, 0x1.d77b654b82c34p-1,
    0x1.d41d41d41d41dp-1, 0x1.d0cb58f6ec074p-1, 0x1.cd85689039b0bp-1,
    0x1.ca4b3055ee191p-1, 0x1.c71c71c71c71cp-1, 0x1.c3f8f01c3f8f0p-1,
    0x1.c0e070381c0e0p-1, 0x1.bdd2b899406f7p-1, 0x1.bacf914c1bad0p-1,
    0x1.b7d6c3dda338bp-1, 0x1.b4e81b4e81b4fp-1, 0x1.b2036406c80d9p-1,
    0x1.af286bca1af28p-1, 0x1.ac5701ac5701bp-1, 0x1.a98ef606a63bep-1,
    0x1.a6d01a6d01a6dp-1, 0x1.a41a41a41a41ap-1, 0x1.a16d3f97a4b02p-1,
    0x1.9ec8e951033d9p-1, 0x1.9c2d14ee4a102p-1, 0x1.999999999999ap-1,
    0x1.970e4f80cb872p-1, 0x1.948b0fcd6e9e0p-1, 0x1.920fb49d0e229p-1,
    0x1.8f9c18f9c18fap-1, 0x1.8d3018d3018d3p-1, 0x1.8acb90f6bf3aap-1,
    0x1.886e5f0abb04ap-1, 0x1.8618618618618p-1, 0x1.83c977ab2beddp-1,
    0x1.8181818181818p-1, 0x1.7f405fd017f40p-1, 0x1.7d05f417d05f4p-1,
    0x1.7ad2208e0ecc3p-1, 0x1.78a4c8178a4c8p-1, 0x1.767dce434a9b1p-1,
    0x1.745d1745d1746p-1, 0x1.724287f46debcp-1, 0x1.702e05c0b8170p-1,
    0x1.6e1f76b4337c7p-1, 0x1.6c16c16c16c17p-1, 0x1.6a13cd1537290p-1,
    0x1.6816816816817p-1, 0x1.661ec6a5122f9p-1, 0x1.642c8590b2164p-1,
    0x1.623fa77016240p-1, 0x1.6058160581606p-1, 0x1.5e75bb8d015e7p-1,
    0x1.5c9882b931057p-1, 0x1.5ac056b015ac0p-1, 0x1.58ed2308158edp-1,
    0x1.571ed3c506b3ap-1, 0x1.5555555555555p-1, 0x1.5390948f40febp-1,
    0x1.51d07eae2f815p-1, 0x1.5015015015015p-1, 0x1.4e5e0a72f0539p-1,
    0x1.4cab88725af6ep-1, 0x1.4afd6a052bf5bp-1, 0x1.49539e3b2d067p-1,
    0x1.47ae147ae147bp-1, 0x1.460cbc7f5cf9ap-1, 0x1.446f86562d9fbp-1,
    0x1.42d6625d51f87p-1, 0x1.4141414141414p-1, 0x1.3fb013fb013fbp-1,
    0x1.3e22cbce4a902p-1, 0x1.3c995a47babe7p-1, 0x1.3b13b13b13b14p-1,
    0x1.3991c2c187f63p-1, 0x1.3813813813814p-1, 0x1.3698df3de0748p-1,
    0x1.3521cfb2b78c1p-1, 0x1.33ae45b57bcb2p-1, 0x1.323e34a2b10bfp-1,
    0x1.30d190130d190p-1, 0x1.2f684bda12f68p-1, 0x1.2e025c04b8097p-1,
    0x1.2c9fb4d812ca0p-1, 0x1.2b404ad012b40p-1, 0x1.29e4129e4129ep-1,
    0x1.288b01288b013p-1, 0x1.27350b8812735p-1, 0x1.25e22708092f1p-1,
    0x1.2492492492492p-1, 0x1.23456789abcdfp-1, 0x1.21fb78121fb78p-1,
    0x1.20b470c67c0d9p-1, 0x1.1f7047dc11f70p-1, 0x1.1e2ef3b3fb874p-1,
    0x1.1cf06ada2811dp-1, 0x1.1bb4a4046ed29p-1, 0x1.1a7b9611a7b96p-1,
    0x1.19453808ca29cp-1, 0x1.1811811811812p-1, 0x1.16e0689427379p-1,
    0x1.15b1e5f75270dp-1, 0x1.1485f0e0acd3bp-1, 0x1.135c81135c811p-1,
    0x1.12358e75d3033p-1, 0x1.1111111111111p-1, 0x1.0fef010fef011p-1,
    0x1.0ecf56be69c90p-1, 0x1.0db20a88f4696p-1, 0x1.0c9714fbcda3bp-1,
    0x1.0b7e6ec259dc8p-1, 0x1.0a6810a6810a7p-1, 0x1.0953f39010954p-1,
    0x1.0842108421084p-1, 0x1.073260a47f7c6p-1, 0x1.0624dd2f1a9fcp-1,
    0x1.05197f7d73404p-1, 0x1.0410410410410p-1, 0x1.03091b51f5e1ap-1,
    0x1.0204081020408p-1, 0x1.0101010101010p-1,
};
static __constant__ double kLogHi[128] = {
    0x0.0p+0, 0x1.fe02a6b106799p-8, 0x1.fc0a8b0fc03c4p-7,
    0x1.7b91b07d5b126p-6, 0x1.f829b0e7832f8p-6, 0x1.39e87b9febd68p-5,
    0x1.77458f632dcffp-5, 0x1.b42dd711971b9p-5, 0x1.f0a30c01162a8p-5,
    0x1.16536eea37ae3p-4, 0x1.341d7961bd1d0p-4, 0x1.51b073f06183cp-4,
    0x1.6f0d28ae56b4ep-4, 0x1.8c345d6319b23p-4, 0x1.a926d3a4ad562p-4,
    0x1.c5e548f5bc743p-4, 0x1.e27076e2af2eap-4, 0x1.fec9131dbeabcp-4,
    0x1.0d77e7cd08e5bp-3, 0x1.1b72ad52f67a2p-3, 0x1.29552f81ff521p-3,
    0x1.371fc201e8f75p-3, 0x1.44d2b6ccb7d1cp-3, 0x1.526e5e3a1b438p-3,
    0x1.5ff3070a793d6p-3, 0x1.6d60fe719d21bp-3, 0x1.7ab890210d907p-3,
    0x1.87fa06520c911p-3, 0x1.9525a9cf456b6p-3, 0x1.a23bc1fe2b561p-3,
    0x1.af3c94e80bff3p-3, 0x1.bc286742d8cd4p-3, 0x1.c8ff7c79a9a20p-3,
    0x1.d5c216b4fbb94p-3, 0x1.e27076e2af2e8p-3, 0x1.ef0adcbdc5935p-3,
    0x1.fb9186d5e3e29p-3, 0x1.0402594b4d041p-2, 0x1.0a324e27390e2p-2,
    0x1.1058bf9ae4ad4p-2, 0x1.1675cababa60fp-2, 0x1.1c898c16999fbp-2,
    0x1.22941fbcf7966p-2, 0x1.2895a13de86a4p-2, 0x1.2e8e2bae11d31p-2,
    0x1.347dd9a987d56p-2, 0x1.3a64c556945eap-2, 0x1.404308686a7e4p-2,
    0x1.4618bc21c5ec2p-2, 0x1.4be5f957778a1p-2, 0x1.51aad872df82ep-2,
    0x1.5767717455a6cp-2, 0x1.5d1bdbf5809cap-2, 0x1.62c82f2b9c796p-2,
    0x1.686c81e9b14adp-2, 0x1.6e08eaa2ba1e4p-2, 0x1.739d7f6bbd007p-2,
    0x1.792a55fdd47a1p-2, 0x1.7eaf83b82afc2p-2, 0x1.842d1da1e8b18p-2,
    0x1.89a3386c1425bp-2, 0x1.8f11e873662c8p-2, 0x1.947941c2116fbp-2,
    0x1.99d958117e08ap-2, 0x1.9f323ecbf984dp-2, 0x1.a484090e5bb09p-2,
    0x1.a9cec9a9a084ap-2, 0x1.af1293247786bp-2, 0x1.b44f77bcc8f64p-2,
    0x1.b9858969310fdp-2, 0x1.beb4d9da71b7ap-2, 0x1.c3dd7a7cdad4dp-2,
    0x1.c8ff7c79a9a21p-2, 0x1.ce1af0b85f3ecp-2, 0x1.d32fe7e00ebd5p-2,
    0x1.d83e7258a2f3ep-2, 0x1.dd46a04c1c4a1p-2, 0x1.e24881a7c6c26p-2,
    0x1.e744261d68789p-2, 0x1.ec399d2468cc1p-2, 0x1.f128f5faf06ecp-2,
    0x1.f6123fa7028adp-2, 0x1.faf588f78f31dp-2, 0x1.ffd2e0857f497p-2,
    0x1.02552a5a5d0ffp-1, 0x1.04bdf9da926d2p-1, 0x1.0723e5c1cdf41p-1,
    0x1.0986f4f573521p-1, 0x1.0be72e4252a83p-1, 0x1.0e44985d1cc8cp-1,
    0x1.109f39e2d4c96p-1, 0x1.12f719593efbdp-1, 0x1.154c3d2f4d5eap-1,
    0x1.179eabbd899a0p-1, 0x1.19ee6b467c96fp-1, 0x1.1c3b81f713c25p-1,
    0x1.1e85f5e7040d1p-1, 0x1.20cdcd192ab6ep-1, 0x1.23130d7bebf43p-1,
    0x1.2555bce98f7cap-1, 0x1.2795e1289b11bp-1, 0x1.29d37fec2b08bp-1,
    0x1.2c0e9ed448e8cp-1, 0x1.2e47436e40268p-1, 0x1.307d7334f10bep-1,
    0x1.32b1339121d71p-1, 0x1.34e289d9ce1d2p-1, 0x1.37117b54747b6p-1,
    0x1.393e0d3562a1ap-1, 0x1.3b68449fffc23p-1, 0x1.3d9026a7156fbp-1,
    0x1.3fb5b84d16f43p-1, 0x1.41d8fe84672afp-1, 0x1.43f9fe2f9ce67p-1,
    0x1.4618bc21c5ec2p-1, 0x1.48353d1ea88dfp-1, 0x1.4a4f85db03ebbp-1,
    0x1.4c679afccee39p-1, 0x1.4e7d811b75bb0p-1, 0x1.50913cc01686bp-1,
    0x1.52a2d265bc5abp-1, 0x1.54b2467999498p-1, 0x1.56bf9d5b3f399p-1,
    0x1.58cadb5cd7989p-1, 0x1.5ad404c359f2dp-1, 0x1.5cdb1dc6c1765p-1,
    0x1.5ee02a9241676p-1, 0x1.60e32f44788d9p-1,
};
static __constant__ double kLogLo[128] = {
    0x0.0p+0, -0x1.e44b7e3711e7fp-67, -0x1.83092c5964281p-62,
    -0x1.6d80ab38e9430p-62, 0x1.33e3f04f1ef25p-60, -0x1.5bfa937f551b7p-59,
    0x1.8d3ca87b92968p-63, 0x1.0a34531f67db5p-59, 0x1.85f325c5bbacdp-59,
    0x1.2189705cf74cap-58, -0x1.3599f227becbbp-58, -0x1.5b61c65e5741ap-58,
    -0x1.20db323097324p-59, -0x1.294d2f5668495p-58, -0x1.d7a16eab1e2adp-59,
    0x1.2eb0bf7c0b0d9p-59, -0x1.61578001e015ap-60, -0x1.5746b9981b36cp-58,
    0x1.9a5dc5e9030adp-57, -0x1.fbe7ee5c69946p-57, 0x1.301771c407dc0p-57,
    0x1.e6cb62af18a02p-62, 0x1.7d3d950f87e23p-59, -0x1.546ff8a470d3ap-57,
    -0x1.bc60efafc6f6cp-58, 0x1.d551d97132e87p-57, -0x1.1072534a57e7dp-57,
    -0x1.9f7fdbfa08d9ap-57, -0x1.26fb3e2b1d1dap-57, 0x1.24dc46c1ea664p-57,
    0x1.a3398064df33ep-57, 0x1.cfce744870f57p-58, -0x1.4f689f8434011p-57,
    -0x1.a37794d03657dp-58, -0x1.61578001e015ep-59, 0x1.e8637950dc20dp-57,
    0x1.355519b0de535p-57, -0x1.08ec217a5022dp-57, 0x1.bdcfde8061c03p-56,
    0x1.3f415699663ecp-63, 0x1.ce63eab883727p-61, 0x1.9f1a39d500e3cp-56,
    -0x1.dbd7ac258a2bdp-58, 0x1.7ad24c13f040fp-56, -0x1.1e99b72bd7bf2p-57,
    -0x1.16ea62c048cfbp-56, 0x1.cbcd735d03424p-60, -0x1.f79f6c1059cdbp-57,
    -0x1.7a42642661c62p-61, -0x1.4b366b609027ap-58, -0x1.d8db0a7cc1543p-56,
    -0x1.fb2a49af933e8p-57, -0x1.7dc9c7c23801fp-56, -0x1.090a0dd59fe35p-58,
    0x1.710af840538e3p-56, -0x1.bfb1b39ca3a0fp-56, 0x1.ce24c53fad3f0p-58,
    0x1.f057691fe9ed7p-56, -0x1.698b43096b576p-59, 0x1.54ec519784677p-56,
    0x1.2d38c40881e0bp-57, 0x1.f85da755a61a3p-56, 0x1.1266e8a3e8838p-57,
    -0x1.315b444ee1f38p-56, -0x1.a92e513217f58p-59, 0x1.fff29adc3ad3bp-56,
    -0x1.ab7b00ad0dabcp-58, 0x1.533844a15dc28p-58, -0x1.a0892a8b38eedp-61,
    -0x1.f3827583b8877p-57, 0x1.be1874deaef08p-56, 0x1.7d9e0a5bd4d37p-57,
    0x1.3097607bcbfeep-56, -0x1.6416a1aa97b31p-57, 0x1.4ef6465f5f46ep-57,
    0x1.c515ba2ec9444p-58, -0x1.19d95b62e2476p-62, 0x1.05ec7a2caa523p-57,
    0x1.cdf68dbcf2ed3p-56, -0x1.94623581958cfp-59, -0x1.328df13bb38c2p-56,
    0x1.5456c3cb6cd06p-58, 0x1.cd7d9f2754362p-57, -0x1.4d05f9366f27fp-59,
    0x1.e9c695d7ee800p-57, 0x1.8fe60804593bfp-56, -0x1.6a1a71dbba44ep-59,
    -0x1.37012b5805e02p-56, 0x1.b4c4bdd99efffp-56, -0x1.c546885a5a707p-59,
    0x1.f78fb26c2de46p-55, -0x1.67f6e731c1795p-56, 0x1.98f33a3965e29p-57,
    -0x1.c73e320bf059fp-58, -0x1.fa3422887e218p-57, -0x1.0b583899021d1p-56,
    -0x1.084e99683070ep-55, -0x1.aabf0bc229014p-55, -0x1.748725e374d6ep-55,
    0x1.9810eb6b440f4p-55, 0x1.ade0fcf6e5a1dp-55, 0x1.01735b2e9733fp-55,
    -0x1.8a158f3917586p-55, 0x1.0950861a4886bp-55, 0x1.fdac850fab36dp-56,
    0x1.d02ab5b3d916bp-56, 0x1.775c96c42e729p-56, -0x1.808bf6deec882p-55,
    -0x1.38eef67f2483ap-55, 0x1.c63b7b06164dap-55, 0x1.0084c7a15a4f5p-58,
    0x1.0a74ea82e55dfp-56, -0x1.ee6d0cf42e7fap-55, 0x1.e1c9ee6d83b86p-55,
    0x1.e85bd9bd99e3ap-56, -0x1.40a85d133f80bp-55, -0x1.d76102e1644f2p-55,
    -0x1.e971322ce7900p-57, -0x1.5d3d9ea6e9ea8p-55, 0x1.9e59d2d85ab62p-56,
    0x1.73be4578ad97bp-56, 0x1.f4550a2d0f60cp-55, 0x1.11c6217363fcbp-57,
    0x1.624bc9764c22cp-55, 0x1.eca6aa97c08e7p-55, 0x1.47b71e2eb8419p-56,
    -0x1.bca7da80b6f7ep-55, -0x1.58376a5f4b135p-57,
};

// 2^(j/2048) as (hi, lo) pairs: one 16-byte shared-memory load per exponential
static __shared__ double2 s_exp2[2048];
static __shared__ double s_log_inv[128];
static __shared__ double s_log_hi[128];
static __shared__ double s_log_lo[128];

// Copies the exp and log tables into this block's shared memory (call before any exp_tang or
// log_tang, with every thread of the block).
__device__ __forceinline__ void exp2_table_init() {
  for (int j = threadIdx.x; j < 2048; j += blockDim.x) {
    s_exp2[j] = make_double2(kExp2Hi[j], kExp2Lo[j]);
  }
  for (int j = threadIdx.x; j < 128; j += blockDim.x) {
    s_log_inv[j] = kLogInv[j];
    s_log_hi[j] = kLogHi[j];
    s_log_lo[j] = kLogLo[j];
  }
  __syncthreads();
}

__device__ __forceinline__ double log_tang(double x) {
  constexpr double kLn2Hi = 0x1.62e42fefa3800p-1, kLn2Lo = 0x1.ef35793c76730p-45;
  const int hi = __double2hiint(x);
  if (hi < 0x00100000 || hi >= 0x7ff00000) return log(x);   // not a positive normal number
  const int lo = __double2loint(x);
  const double e = (double)((hi >> 20) - 1023);
  const int j = (hi >> 13) & 127;
  const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);
  const double r = fma(m, s_log_inv[j], -1.0);
  double q = fma(r, -1.0 / 8.0, 1.0 / 7.0);
  q = fma(r, q, -1.0 / 6.0);
  q = fma(r, q, 1.0 / 5.0);
  q = fma(r, q, -1.0 / 4.0);
  q = fma(r, q, 1.0 / 3.0);
  q = fma(r, q, -0.5);
  const double small = fma(r * r, q, r) + fma(e, kLn2Lo, s_log_lo[j]);
  return fma(e, kLn2Hi, s_log_hi[j]) + small;
}

__device__ __forceinline__ double exp_tang(double x) {
  constexpr double kInvL = 0x1.71547652b82fep+11;   // 2048 / ln 2
  constexpr double kLhi = 0x1.62e42fefa39efp-12;    // ln 2 / 2048, leading 53 bits
  constexpr double kLlo = 0x1.abc9e3b39803fp-67;    // ln 2 / 2048 - kLhi
  constexpr double kShift = 6755399441055744.0;     // 1.5 * 2^52: round to nearest integer
  const bool in_range = (__double2hiint(x) & 0x7fffffff) < 0x40800000;   // |x| < 512
  const double t = fma(x, kInvL, kShift);
  const double nd = t - kShift;
  const int n = __double2loint(t);
  double r = fma(-nd, kLhi, x);
  r = fma(-nd, kLlo, r);
  const double p = fma(r * r, fma(r, 1.0 / 6.0, kExpC2), r);
  const double2 tt = s_exp2[n & 2047];
  const double th = tt.x, tl = tt.y;
  const double y = th + fma(th, p, tl);
  const int m = n >> 11;   // floor(n / 2048): n = 2048 m + (n & 2047)
  const double out =
      __hiloint2double(__double2hiint(y) + (int)((unsigned)m << 20), __double2loint(y));
  return in_range ? out : exp(x);
}

// 2^y, the same table method in base 2: y = (2048 m + j)/2048 + r with |r| <= 2^-12 exactly (no
// split constant: 2048 y and n/2048 are exact), 2^y = 2^m * 2^(j/2048) * 2^r.  Eight FP64
// instructions.  The ionic kernel's exponentials exp(c x) are 2^((c log2 e) x) with the factor
// folded into the constant c, so the change of base costs nothing at the call sites.  |y| >= 704,
// inf and NaN go to the library exp2.
__device__ __forceinline__ double exp2_tang(double y) {
  constexpr double kShift = 6755399441055744.0;   // 1.5 * 2^52: round to nearest integer
  const bool in_range = (__double2hiint(y) & 0x7fffffff) < 0x40860000;   // |y| < 704
  const double t = fma(y, 2048.0, kShift);
  const double nd = t - kShift;
  const int n = __double2loint(t);
  const double r = fma(-nd, 1.0 / 2048.0, y);
  const double p = r * fma(r, fma(r, kExp2A3, kExp2A2), kExp2A1);
  const double2 tt = s_exp2[n & 2047];
  const double th = tt.x, tl = tt.y;
  const double out0 = th + fma(th, p, tl);
  const int m = n >> 11;
  const double out =
      __hiloint2double(__double2hiint(out0) + (int)((unsigned)m << 20), __double2loint(out0));
  return in_range ? out : exp2(y);
}

// 1/d for a finite, nonzero, normal d: the hardware estimate (rcp.approx, relative error below
// 2^-20) refined by two Newton-Raphson steps y <- y + y (1 - d y), each of which squares the
// relative error.  Four FP64 instructions against about twice that for a division; on 2.7 M
// sampled d in [1e-20, 1e20] it matched the correctly rounded 1/d in every case.
__device__ __forceinline__ double rcp_estimate(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  return y;
}

__device__ __forceinline__ double rcp_nr(double d) {
  double y = rcp_estimate(d);
  double e = fma(-d, y, 1.0);
  y = fma(y, e, y);
  e = fma(-d, y, 1.0);
  return fma(y, e, y);
}

__device__ __forceinline__ double mexp(double x) { return exp_tang(x); }
__device__ __forceinline__ float mexp(float x) { return expf(x); }
__device__ __forceinline__ double mexp2(double y) { return exp2_tang(y); }
__device__ __forceinline__ float mexp2(float y) { return exp2f(y); }
// c x + d as one FMA (exponent arguments c (x + a) are written with d = a c folded at compile time)
template <typename T>
__device__ __forceinline__ T affine(T x, double c, double d) { return fmaT(x, T(c), T(d)); }
// c (x + b)^2 = (c x + 2 b c) x + b^2 c: two FMAs
template <typename T>
__device__ __forceinline__ T gauss_arg(T x, double c, double b) { return fmaT(x, fmaT(x, T(c), T(2 * b * c)), T(b * b * c)); }
__device__ __forceinline__ double mlog(double x) { return log_tang(x); }
__device__ __forceinline__ float mlog(float x) { return logf(x); }
__device__ __forceinline__ double mrcp(double x) { return rcp_nr(x); }
__device__ __forceinline__ float mrcp(float x) { return 1.f / x; }
__device__ __forceinline__ double msqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float msqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double mexpm1(double x) { return expm1(x); }
__device__ __forceinline__ float mexpm1(float x) { return expm1f(x); }

// Voltage-only factors shared by the two current evaluations of a step.
template <typename T>
struct Tp06VFactors {
  T ghk;        // L-type driving factor without CaSS: split into a and b so that
  T ghk_cass;   // I_CaL / (g d f f2 fCass) = ghk_cass * CaSS + ghk
  T nak;        // I_NaK / (Nai / (Nai + KmNa))
  T naca_a;     // exp(gamma V F/RT) / denominator * kNaCa
  T naca_b;     // exp((gamma-1) V F/RT) / denominator * kNaCa * alpha
  T ipk;        // 1 / (1 + exp((25 - V)/5.98))
};

template <typename T>
__device__ __forceinline__ Tp06VFactors<T> tp06_vfactors(T V) {
  using namespace tp06;
  Tp06VFactors<T> f;
  const T vf2 = V * T(kLog2e / kRTF);         // V F/RT log2 e
  const T q = mexp2(-vf2);                     // exp(-V F/RT)
  const T eg = mexp2(T(kGam) * vf2);
  const T eg1 = eg * q;                        // exp((gamma - 1) V F/RT)
  const T vm = V - T(15);
  const T x = vm * T(2.0 / kRTF);
  if (fabs(x) >= T(0.5)) {
    // exp(x) = K / q^2 with K = exp(-30 F/RT), so that both GHK factors share the denominator
    // K - q^2 (exp(x) - 1 times q^2), which keeps its relative accuracy while |x| >= 1/2
    const T q2 = q * q;
    const T sg = vm * T(kF / kRTF) * mrcp(T(kGhkK) - q2);
    f.ghk_cass = sg * T(kGhkK);
    f.ghk = T(-4 * kCao) * sg * q2;
  } else if (x != T(0)) {   // within 6.7 mV of 15 mV: the library expm1
    const T em1 = mexpm1(x);
    const T c = T(4) * vm * T(kF / kRTF) / em1;
    f.ghk_cass = c * T(0.25) * (em1 + T(1));
    f.ghk = -c * T(kCao);
  } else {   // limit V -> 15 mV: 2 F (0.25 CaSS - Cao)
    f.ghk_cass = T(2 * kF * 0.25);
    f.ghk = T(-2 * kF * kCao);
  }
  // I_NaK, I_NaCa and I_pK factors: three quotients over one reciprocal of their denominators
  const T dn = T(1) + T(0.1245) * mexp2(T(-0.1) * vf2) + T(0.0353) * q;
  const T den = T((kKmNai * kKmNai * kKmNai + kNao * kNao * kNao) * (kKmCa + kCao)) *
                (T(1) + T(kKsat) * eg1);
  const T dp = T(1) + mexp2(affine(V, -kLog2e / 5.98, 25 * kLog2e / 5.98));
  const T rr = mrcp(dn * den * dp);
  f.nak = T(kPNaK * kKo / (kKo + kKmK)) * (den * dp * rr);
  const T rden = dn * dp * rr;
  f.naca_a = T(kKNaCa) * eg * rden;
  f.naca_b = T(kKNaCa * kAlphaNaCa * kNao * kNao * kNao) * eg1 * rden;
  f.ipk = dn * den * rr;
  return f;
}

template <typename T>
struct Tp06Currents {
  T ik;    // I_K1 + I_to + I_Kr + I_pK (all through V - E_K)
  T ina;   // I_Na + I_bNa (both through V - E_Na)
  T iks, inak, inaca, ical, ibca, ipca;
  __device__ __forceinline__ T total() const { return ik + ina + iks + ical + ibca + inak + inaca + ipca; }
};

// The concentration-dependent transcendental part of a current evaluation: the logarithms of the
// Nernst potentials' concentrations and the exponentials of I_K1 at dv = V - E_K.
template <typename T>
struct Tp06Nernst {
  T lki, lnai, lks, lcai;   // ln Ki, ln Nai, ln(Ki + pKNa Nai), ln Cai
  T dv;                     // V - E_K
  T ea, eb, e3, e10;        // exp(0.06 (dv - 200)), exp(-0.5 dv), exp(0.0002 (dv + 100)), exp(0.1 (dv - 10))
};

template <typename T>
__device__ __forceinline__ void tp06_k1_exps(Tp06Nernst<T>& n) {
  n.ea = mexp2(affine(n.dv, 0.06 * kLog2e, -200 * 0.06 * kLog2e));
  n.eb = mexp2(T(-0.5 * kLog2e) * n.dv);
  n.e3 = mexp2(affine(n.dv, 0.0002 * kLog2e, 100 * 0.0002 * kLog2e));
  n.e10 = mexp2(affine(n.dv, 0.1 * kLog2e, -10 * 0.1 * kLog2e));
}

// Nernst potentials as differences of logarithms (the constants' logarithms folded at compile
// time), which saves the divisions of the quotient forms
template <typename T>
__device__ __forceinline__ Tp06Nernst<T> tp06_nernst(T V, const T* u) {
  using namespace tp06;
  Tp06Nernst<T> n;
  n.lki = mlog(u[0]);
  n.lnai = mlog(u[1]);
  n.lks = mlog(u[0] + T(kPKNa) * u[1]);
  n.lcai = mlog(u[2]);
  n.dv = V - T(kRTF) * (T(kLnKo) - n.lki);
  tp06_k1_exps(n);
  return n;
}

// The same after one step of the slow concentrations, from the evaluation before it: Ki and Nai
// change by about 1e-7 of their value per step, so ln x' = ln x + log1p(t), t = (x' - x)/x, with
// log1p(t) = t - t^2/2 + t^3/3 (error below t^4/4 < 2^-82 for |t| < 2^-20; t needs only 31
// correct bits there, which one Newton step on the reciprocal estimate gives), and
// exp(a dv') = exp(a dv) exp(a e), e = dv' - dv, with exp(z) = 1 + z + z^2/2 + z^3/6 (error below
// z^4/24 < 2^-55 relative for |e| < 2^-12).  Larger changes take the full evaluation.  Cai
// (several per cent per step in an upstroke) always takes the table log.
__device__ __forceinline__ double log1p_small(double t) { return fma(t * t, fma(t, 1.0 / 3.0, -0.5), t); }
__device__ __forceinline__ double exp_small(double z) { return fma(z, fma(z, fma(z, 1.0 / 6.0, 0.5), 1.0), 1.0); }
__device__ __forceinline__ double rel_change(double x0, double x1) {
  const double y = rcp_estimate(x0);
  return (x1 - x0) * fma(y, fma(-x0, y, 1.0), y);
}

__device__ __forceinline__ Tp06Nernst<double> tp06_nernst_next(double V, const double* u1, double ki0, double nai0,
                                                               const Tp06Nernst<double>& n0) {
  using namespace tp06;
  const double ks0 = ki0 + kPKNa * nai0, ks1 = u1[0] + kPKNa * u1[1];
  const double tk = rel_change(ki0, u1[0]), tn = rel_change(nai0, u1[1]), ts = rel_change(ks0, ks1);
  constexpr double kT = 0x1p-20;
  if (!(fabs(tk) < kT && fabs(tn) < kT && fabs(ts) < kT)) return tp06_nernst(V, u1);
  Tp06Nernst<double> n;
  n.lki = n0.lki + log1p_small(tk);
  n.lnai = n0.lnai + log1p_small(tn);
  n.lks = n0.lks + log1p_small(ts);
  n.lcai = mlog(u1[2]);
  n.dv = V - kRTF * (kLnKo - n.lki);
  const double e = n.dv - n0.dv;
  if (!(fabs(e) < 0x1p-12)) {
    tp06_k1_exps(n);
    return n;
  }
  n.ea = n0.ea * exp_small(0.06 * e);
  n.eb = n0.eb * exp_small(-0.5 * e);
  n.e3 = n0.e3 * exp_small(0.0002 * e);
  n.e10 = n0.e10 * exp_small(0.1 * e);
  return n;
}

// The same from logarithms held over from the previous step (lg: ln Ki, ln Nai, ln(Ki + pKNa Nai),
// ln Cai of the current states, computed by tp06_nernst_next_direct at the end of that step).
template <typename T>
__device__ __forceinline__ Tp06Nernst<T> tp06_nernst_logs(T V, const T* lg) {
  using namespace tp06;
  Tp06Nernst<T> n;
  n.lki = lg[0];
  n.lnai = lg[1];
  n.lks = lg[2];
  n.lcai = lg[3];
  n.dv = V - T(kRTF) * (T(kLnKo) - n.lki);
  tp06_k1_exps(n);
  return n;
}

// After the states' step: the logarithms directly (so that the next step can take them as they
// are and still agree bit for bit with a step that computes them) and the I_K1 exponentials
// carried over from the evaluation before the step when dv moved by less than 2^-12 (as in
// tp06_nernst_next).
__device__ __forceinline__ Tp06Nernst<double> tp06_nernst_next_direct(double V, const double* u1,
                                                                      const Tp06Nernst<double>& n0) {
  using namespace tp06;
  Tp06Nernst<double> n;
  n.lki = mlog(u1[0]);
  n.lnai = mlog(u1[1]);
  n.lks = mlog(u1[0] + kPKNa * u1[1]);
  n.lcai = mlog(u1[2]);
  n.dv = V - kRTF * (kLnKo - n.lki);
  const double e = n.dv - n0.dv;
  if (!(fabs(e) < 0x1p-12)) {
    tp06_k1_exps(n);
    return n;
  }
  n.ea = n0.ea * exp_small(0.06 * e);
  n.eb = n0.eb * exp_small(-0.5 * e);
  n.e3 = n0.e3 * exp_small(0.0002 * e);
  n.e10 = n0.e10 * exp_small(0.1 * e);
  return n;
}

template <typename T>
__device__ __forceinline__ Tp06Currents<T> tp06_currents(T V, const T* u, int cell, const Tp06VFactors<T>& f,
                                                         const Tp06Nernst<T>& n) {
  using namespace tp06;
  const T nai = u[1], cai = u[2], cass = u[4];
  const T ena = T(kRTF) * (T(kLnNao) - n.lnai);
  const T eks = T(kRTF) * (T(kLnKsNa) - n.lks);
  const T eca = T(0.5 * kRTF) * (T(kLnCao) - n.lcai);
  const T dv = n.dv;
  // alpha_K1 / (alpha_K1 + beta_K1) over one common denominator
  const T nb = T(3) * n.e3 + n.e10;
  const T na = T(0.1) * (T(1) + n.eb);
  // the quotients of I_K1, I_NaK and I_pCa over one reciprocal of their denominators
  const T d1 = na + nb * (T(1) + n.ea), d2 = nai + T(kKmNa), d3 = T(kKpCa) + cai;
  const T d23 = d2 * d3;
  const T rr = mrcp(d1 * d23);
  Tp06Currents<T> c;
  const T gto = cell == 0 ? T(0.073) : T(0.294);
  const T gks = cell == 1 ? T(0.098) : T(0.392);
  // the currents that share a driving force as one conductance sum times it: I_K1 (with
  // sqrt(Ko/5.4) = 1 at Ko = 5.4 mM), I_to, I_Kr and I_pK through V - E_K; I_Na and I_bNa
  // through V - E_Na
  const T gk = fmaT(T(kGKr) * u[6], u[7], fmaT(gto * u[17], u[16], fmaT(T(kGK1) * na, d23 * rr, T(kGpK) * f.ipk)));
  c.ik = gk * dv;
  const T m = u[9];
  c.ina = fmaT(T(kGNa) * m * m * m * u[10], u[11], T(kGbNa)) * (V - ena);
  c.iks = gks * u[8] * u[8] * (V - eks);
  c.ical = T(kGCaL) * u[12] * u[13] * u[14] * u[15] * (f.ghk_cass * cass + f.ghk);
  c.ibca = T(kGbCa) * (V - eca);
  c.inak = f.nak * nai * (d1 * d3 * rr);
  c.inaca = f.naca_a * (nai * nai * nai) * T(kCao) - f.naca_b * cai;
  c.ipca = T(kGpCa) * cai * (d1 * d2 * rr);
  return c;
}

// Rush-Larsen update of one gate, u_inf + (u - u_inf) exp(-dt/tau), with the gate's rate
// 1/tau given (no division) and dtl = dt log2 e (exp(-dt rate) = 2^(-dtl rate)).
template <typename T>
__device__ __forceinline__ T rl_rate(T u, T inf, T rate, T dtl) {
  return inf + (u - inf) * mexp2(-dtl * rate);
}

// The same for a slow gate, whose tau has a lower bound over every V (x_s 80 ms, f 98.8 ms, f2
// 8.79 ms, the last at V = 11.4 mV): for dt <= 0.025 ms, z = dt/tau <= 2.9e-3 and exp(-z) is its
// degree-5 Taylor polynomial (error below z^6/720 < 1e-18); other steps take the exponential.
template <typename T>
__device__ __forceinline__ T rl_rate_slow(T u, T inf, T rate, T dt, T dtl, bool short_step) {
  T e;
  if (short_step) {
    const T z = dt * rate;
    e = fmaT(z, fmaT(z, fmaT(z, fmaT(z, fmaT(z, T(-1.0 / 120.0), T(1.0 / 24.0)), T(-1.0 / 6.0)), T(0.5)), T(-1.0)), T(1.0));
  } else {
    e = mexp2(-dtl * rate);
  }
  return inf + (u - inf) * e;
}

// One operator-split step of a single cell: u (18 states, in/out) advances from (V, u^k) to
// u^{k+1}; returns I_ion(V, u^{k+1}) in pA/pF.  With lg (FP64), the four concentration
// logarithms are held across steps: read from lg at the start when lg_valid, written to lg for
// u^{k+1} at the end.
template <typename T>
__device__ __forceinline__ T tp06_cell_step(T V, T* u, int cell, T dt, T* lg = nullptr, bool lg_valid = false) {
  using namespace tp06;
  const Tp06VFactors<T> vf = tp06_vfactors(V);
  const Tp06Nernst<T> nern = lg && lg_valid ? tp06_nernst_logs(V, lg) : tp06_nernst(V, u);
  const Tp06Currents<T> c = tp06_currents(V, u, cell, vf, nern);

  // concentrations and Rbar: forward Euler from the rates at (V^k, u^k)
  T un[kTP06States];
  {
    const T cai = u[2], casr = u[3], cass = u[4], rbar = u[5];
    // the same expressions with each quotient of quotients over one denominator
    // six quotients, two reciprocals: k_casr with I_up, then O with the three buffer factors
    const T casr2 = casr * casr, cai2 = cai * cai;
    const T dk = casr2 + T(kEC * kEC), du = cai2 + T(kKup * kKup);
    const T r1 = mrcp(dk * du);
    const T kcasr = T(kMaxSR) - T(kMaxSR - kMinSR) * casr2 * (du * r1);
    const T iup = T(kVmaxUp) * cai2 * (dk * r1);
    const T k2 = T(kK2p) * kcasr;
    const T cass2 = cass * cass;
    const T bi = cai + T(kKbufc), bsr = casr + T(kKbufsr), bss = cass + T(kKbufss);
    const T bi2 = bi * bi, bsr2 = bsr * bsr, bss2 = bss * bss;
    const T dox = T(kK3) * kcasr + T(kK1p) * cass2, dfi = bi2 + T(kBufc * kKbufc);
    const T dsr = bsr2 + T(kBufsr * kKbufsr), dss = bss2 + T(kBufss * kKbufss);
    const T pa = dox * dfi, pb = dsr * dss;
    const T r2 = mrcp(pa * pb);
    const T o = T(kK1p) * cass2 * rbar * (dfi * pb * r2);
    const T irel = T(kVrel) * o * (casr - cass);
    const T ileak = T(kVleak) * (casr - cai);
    const T ixfer = T(kVxfer) * (cass - cai);
    const T fi = bi2 * (dox * pb * r2);
    const T fsr = bsr2 * (pa * dss * r2);
    const T fss = bss2 * (pa * dsr * r2);
    const T cvf = T(kCap / (kVc * kF));
    const T dki = -(c.ik + c.iks - T(2) * c.inak) * cvf;
    const T dnai = -(c.ina + T(3) * (c.inak + c.inaca)) * cvf;
    const T dcai = fi * ((ileak - iup) * T(kVsr / kVc) + ixfer -
                         (c.ibca + c.ipca - T(2) * c.inaca) * T(kCap / (2 * kVc * kF)));
    const T dcasr = fsr * (iup - (irel + ileak));
    const T dcass = fss * (-c.ical * T(kCap / (2 * kVss * kF)) + irel * T(kVsr / kVss) -
                           ixfer * T(kVc / kVss));
    const T drbar = -k2 * cass * rbar + T(kK4) * (T(1) - rbar);
    un[0] = u[0] + dt * dki;
    un[1] = u[1] + dt * dnai;
    un[2] = cai + dt * dcai;
    un[3] = casr + dt * dcasr;
    un[4] = cass + dt * dcass;
    un[5] = rbar + dt * drbar;
  }
  // gates: Rush-Larsen with inf and tau at V^k (fCass at CaSS^k).  Each rate 1/tau is formed
  // directly over one common denominator, and a gate's steady state and rate share one reciprocal
  // of the product of their denominators (one division per gate); divisions by constants are
  // multiplications by reciprocals.  Exponentials exp(a V + b) whose slope a is shared (or is
  // minus, or minus twice, a shared slope) are the shared exp(a V) times literal exp(b).
  {
    const T dtl = dt * T(kLog2e);
    const bool short_step = dt <= T(0.025);
    // exp(-V/20), exp(-V/10) = its square, exp(V/5) = 1/exp(-V/10)^2: one exponential for three
    const T xm005 = mexp2(T(-0.05 * kLog2e) * V);
    const T xm01 = xm005 * xm005;                    // exp(-V/10)
    const T x02 = mrcp(xm01 * xm01);                 // exp(V/5)
    const T xm16 = mexp2(V * T(-kLog2e / 6.0));
    const T x17 = mexp2(V * T(kLog2e / 7.0));
    const T y15 = mexp2(V * T(kLog2e / 15.0));
    // m: inf = 1/(1+e1)^2; 1/tau = (1 + e^-12/x02) eb ec / (0.1 (eb + ec))
    //                            = (x02 + e^-12) eb ec / (0.1 x02 (eb + ec))
    {
      const T e1 = T(1) + mexp2(affine(V, -kLog2e / 9.03, -56.86 * kLog2e / 9.03));
      const T p1 = e1 * e1;
      const T eb = T(1) + x02 * T(kE7);
      const T ec = T(1) + mexp2(affine(V, kLog2e / 200.0, -50 * kLog2e / 200.0));
      const T qm = T(0.1) * x02 * (eb + ec);
      const T r = mrcp(p1 * qm);
      un[9] = rl_rate(u[9], qm * r, (x02 + T(kEm12)) * eb * ec * p1 * r, dtl);
    }
    // h and j: inf = 1/(1+e2)^2 for both; rates alpha + beta
    {
      const T e2 = T(1) + mexp2(affine(V, kLog2e / 7.43, 71.55 * kLog2e / 7.43));
      const T p2 = e2 * e2;
      T hinf, rh, rj;
      if (V < T(-40)) {
        rh = T(0.057) * mexp2(affine(V, -kLog2e / 6.8, -80 * kLog2e / 6.8)) + T(2.7) * mexp2(T(0.079 * kLog2e) * V) +
             T(3.1e5) * mexp2(T(0.3485 * kLog2e) * V);
        const T ja = T(1) + mexp2(affine(V, 0.311 * kLog2e, 79.23 * 0.311 * kLog2e));
        const T jb = T(1) + mexp2(affine(V, -0.1378 * kLog2e, -40.14 * 0.1378 * kLog2e));
        const T jab = ja * jb;
        const T r = mrcp(p2 * jab);
        hinf = jab * r;
        rj = ((T(-2.5428e4) * mexp2(T(0.2444 * kLog2e) * V) - T(6.948e-6) * mexp2(T(-0.04391 * kLog2e) * V)) * (V + T(37.78)) * jb +
              T(0.02424) * mexp2(T(-0.01052 * kLog2e) * V) * ja) *
             p2 * r;
      } else {
        const T dh = T(1) + mexp2(affine(V, -kLog2e / 11.1, -10.66 * kLog2e / 11.1));
        const T dj = T(1) + xm01 * T(kEm3p2);
        const T dhj = dh * dj;
        const T r = mrcp(p2 * dhj);
        hinf = dhj * r;
        rh = T(0.77 / 0.13) * p2 * dj * r;
        rj = T(0.6) * mexp2(T(0.057 * kLog2e) * V) * p2 * dh * r;
      }
      un[10] = rl_rate(u[10], hinf, rh, dtl);
      un[11] = rl_rate(u[11], hinf, rj, dtl);
    }
    // xr1 and xr2: xr1_inf = 1/(1 + e^(-26/7)/x17) = x17/(x17 + e^(-26/7)), xr2_inf = 1/(1+e);
    // 1/tau_xr1 = (1+e)(1+e')/2700; 1/tau_xr2 = (1 + xm005 e^-3)(1 + e^-3/xm005)/3.36
    //                                         = (1 + xm005 e^-3)(xm005 + e^-3)/(3.36 xm005)
    {
      const T a1 = x17 + T(kEm26o7);
      const T b2 = T(1) + mexp2(affine(V, kLog2e / 24.0, 88 * kLog2e / 24.0));
      const T a1b2 = a1 * b2;
      const T r = mrcp(a1b2 * xm005);
      un[6] = rl_rate(u[6], x17 * b2 * xm005 * r,
                      (T(1) + xm01 * T(kEm4p5)) * (T(1) + mexp2(affine(V, kLog2e / 11.5, 30 * kLog2e / 11.5))) *
                          T(1.0 / 2700.0),
                      dtl);
      un[7] = rl_rate(u[7], a1 * xm005 * r,
                      (T(1) + xm005 * T(kEm3)) * (xm005 + T(kEm3)) * a1b2 * r * T(1.0 / 3.36), dtl);
    }
    // xs: tau = 1400/(sqrt(1+e)(1+e')) + 80, so 1/tau = sx/(1400 + 80 sx)
    {
      const T axs = T(1) + mexp2(affine(V, -kLog2e / 14.0, -5 * kLog2e / 14.0));
      const T sx = msqrt(T(1) + xm16 * T(kE5o6)) * (T(1) + y15 * T(kEm35o15));
      const T bxs = T(1400) + T(80) * sx;
      const T r = mrcp(axs * bxs);
      un[8] = rl_rate_slow(u[8], bxs * r, sx * axs * r, dt, dtl, short_step);
    }
    // r: inf = 1/(1 + xm16 e^(20/6)), tau = 9.5 exp(-(V+40)^2/1800) + 0.8
    {
      const T ar = T(1) + xm16 * T(kE20o6);
      const T br = T(9.5) * mexp2(gauss_arg(V, -kLog2e / 1800.0, 40.0)) + T(0.8);
      const T r = mrcp(ar * br);
      un[17] = rl_rate(u[17], br * r, ar * r, dtl);
    }
    // s (endocardial: tau = 1000 exp(-(V+67)^2/1000) + 8; else tau = 85 e + 5/(1+e') + 3)
    {
      T as, bs, ns;
      if (cell == 0) {
        as = T(1) + x02 * T(kE5p6);
        bs = T(1000) * mexp2(gauss_arg(V, -kLog2e / 1000.0, 67.0)) + T(8);
        ns = T(1);
      } else {
        as = T(1) + x02 * T(kE4);
        ns = T(1) + x02 * T(kEm4);
        bs = (T(85) * mexp2(gauss_arg(V, -kLog2e / 320.0, 45.0)) + T(3)) * ns + T(5);
      }
      const T r = mrcp(as * bs);
      un[16] = rl_rate(u[16], bs * r, ns * as * r, dtl);
    }
    // d: inf = 1/(1 + e^(-8/7.5)/y15^2) = y15^2/(y15^2 + e^(-8/7.5));
    // tau = (1.4/(1+ea) + 0.25) 1.4/(1+eb) + 1/(1+ec)
    {
      const T y2 = y15 * y15;
      const T ad = y2 + T(kEm8o7p5);
      const T da = T(1) + mexp2(affine(V, -kLog2e / 13.0, -35 * kLog2e / 13.0));
      const T db = T(1) + x02 * T(kE1);
      const T dc = T(1) + xm005 * T(kE2p5);
      const T bd = (T(1.4) + T(0.25) * da) * T(1.4) * dc + da * db;
      const T r = mrcp(ad * bd);
      un[12] = rl_rate(u[12], y2 * bd * r, da * db * dc * ad * r, dtl);
    }
    // f and f2 share fb = 1 + exp((V+30)/10) = F/xm01 with F = xm01 + e^3;
    // tau_f = 1102.5 g + 200/(1+ea) + 180/(1+fb) + 20, tau_f2 = 562 g' + 31/(1+ga) + 80/(1+fb)
    // with g = exp(-(V+27)^2/225), g' = exp(-(V+27)^2/240)
    const T F = xm01 + T(kE3);
    {
      const T af = T(1) + x17 * T(kE20o7);
      const T fa = T(1) + xm01 * T(kE1p3);
      const T num = (T(1102.5) * mexp2(gauss_arg(V, -kLog2e / 225.0, 27.0)) + T(20)) * fa * F + T(200) * F +
                    T(180) * fa * xm01;
      const T r = mrcp(af * num);
      un[13] = rl_rate_slow(u[13], num * r, fa * F * af * r, dt, dtl, short_step);
    }
    {
      const T af2 = T(1) + x17 * T(kE5);
      const T ga = T(1) + xm01 * T(kE2p5);
      const T num = T(562) * mexp2(gauss_arg(V, -kLog2e / 240.0, 27.0)) * ga * F + T(31) * F + T(80) * ga * xm01;
      const T r = mrcp(af2 * num);
      un[14] = rl_rate_slow(u[14], T(0.67) * num * r + T(0.33), ga * F * af2 * r, dt, dtl, short_step);
    }
    // fCass: inf = 0.6 q + 0.4, 1/tau = 1/(80 q + 2) = s2/(80 + 2 s2), q = 1/s2, s2 = 1 + (CaSS/0.05)^2
    {
      const T cs = u[4] * T(20);
      const T s2 = T(1) + cs * cs;
      const T b = T(80) + T(2) * s2;
      const T r = mrcp(s2 * b);
      un[15] = rl_rate(u[15], T(0.6) * (b * r) + T(0.4), s2 * s2 * r, dtl);
    }
  }
  // I_ion at (V^k, u^{k+1}); FP64 carries the slow concentrations' logarithms over (see above)
  Tp06Nernst<T> nern1;
  if constexpr (sizeof(T) == 8) {
    if (lg) {
      nern1 = tp06_nernst_next_direct(V, un, nern);
      lg[0] = nern1.lki;
      lg[1] = nern1.lnai;
      lg[2] = nern1.lks;
      lg[3] = nern1.lcai;
    } else {
      nern1 = tp06_nernst_next(V, un, u[0], u[1], nern);
    }
  } else {
    nern1 = tp06_nernst(V, un);
  }
  const T iion = tp06_currents(V, un, cell, vf, nern1).total();
#pragma unroll
  for (int j = 0; j < kTP06States; ++j) u[j] = un[j];
  return iion;
}

// (a1) Ionic update of the tissue, TP06.  With a learned surrogate attached, nodes flagged for it
// carry the window's effective current instead (their states already hold the surrogate's
// end-of-window prediction); all other nodes take the exact step.
// Launch shape per precision (measured on the 40x16x6 mm slab).  FP64: 128-thread blocks, four
// per SM (16 warps, 128 registers, no spill) - 2.5 % faster than two 256-thread blocks with the
// same warps; five or six per SM (fewer registers, spills) were slower.  FP32: 256-thread blocks, three per SM
// (10 % slower at 128 x 5).
template <typename T>
struct Tp06Launch {
  static constexpr int threads = 128, min_blocks = 8;
};
template <>
struct Tp06Launch<double> {
  static constexpr int threads = 128, min_blocks = 4;
};

template <typename T>
__global__ void __launch_bounds__(Tp06Launch<T>::threads, Tp06Launch<T>::min_blocks)
    ionic_tp06_kernel(const IonicArgs<T> a) {
  // the FP64 exp and log tables; the FP32 kernel uses the hardware exp2f and logf and stages
  // nothing (35 KB of copies per block, and the shared memory they held, saved)
  if constexpr (sizeof(T) == 8) exp2_table_init();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.n_bar) a.bar[i].count = 0u;
  if (i >= a.n) return;
  const int64_t n = a.n;
  const T V = a.V[i], Vp = a.Vp[i];
  T iion;
  if (a.sur_flag && a.sur_flag[i]) {
    iion = T(a.cm) * T(a.sur_iion[i]);
  } else {
    T u[kTP06States];
#pragma unroll
    for (int j = 0; j < kTP06States; ++j) u[j] = a.state[j * n + i];
    // the concentration logarithms of u^k, left by the previous step (FP64, when valid)
    T lg[4];
    const bool cache = a.log_cache != nullptr;
    bool valid = cache && *a.log_valid != 0;
    if (valid) {
#pragma unroll
      for (int q = 0; q < 4; ++q) lg[q] = a.log_cache[q * n + i];
      valid = lg[0] == lg[0];   // NaN: the surrogate replaced this node's states since they were taken
    }
    iion = T(a.cm) * tp06_cell_step(V, u, a.cell, T(a.dt), cache ? lg : nullptr, valid);
#pragma unroll
    for (int j = 0; j < kTP06States; ++j) a.state[j * n + i] = u[j];
    if (cache) {
#pragma unroll
      for (int q = 0; q < 4; ++q) a.log_cache[q * n + i] = lg[q];
    }
  }
  const T is = T(stimulus_at(a.stim_off, a.stim_ids, a.stims, i, *a.k_base + a.k_off));
  rhs_epilogue(a, i, V, Vp, iion, is);
}

// Exact single-cell windows: from (u, V) with a constant stimulus (pA/pF), nsub split steps of
// the cell (states as in the tissue step, then V += dt (I_stim - I_ion)).  Inputs and outputs are
// [19][n] FP32 (18 states, then V); the arithmetic is in T.
template <typename T>
__global__ void __launch_bounds__(256) tp06_window_kernel(int64_t n, const float* in, const float* istim,
                                                        float* out, int cell, double dt, int nsub) {
  exp2_table_init();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T u[kTP06States];
#pragma unroll
  for (int j = 0; j < kTP06States; ++j) u[j] = T(in[j * n + i]);
  T V = T(in[kTP06States * n + i]);
  const T is = istim ? T(istim[i]) : T(0);
  for (int k = 0; k < nsub; ++k) {
    const T iion = tp06_cell_step(V, u, cell, T(dt));
    V = V + T(dt) * (is - iion);
  }
#pragma unroll
  for (int j = 0; j < kTP06States; ++j) out[j * n + i] = float(u[j]);
  out[kTP06States * n + i] = float(V);
}

// Self-test of exp_tang (fn 0) or log_tang (fn 1) against the library function on device
// (diagnostics of the ABI).
static __global__ void __launch_bounds__(256) exp_selftest_kernel(int64_t n, const double* x, double* y_fast,
                                                           double* y_ref, int fn) {
  exp2_table_init();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y_fast[i] = fn == 3 ? exp2_tang(x[i]) : fn == 2 ? rcp_nr(x[i]) : fn == 1 ? log_tang(x[i]) : exp_tang(x[i]);
  y_ref[i] = fn == 3 ? exp2(x[i]) : fn == 2 ? 1.0 / x[i] : fn == 1 ? log(x[i]) : exp(x[i]);
}

}  // namespace tc

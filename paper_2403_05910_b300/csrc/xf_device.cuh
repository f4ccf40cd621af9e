// xf_device.cuh -- sm_103a kernels of the multicomponent RHS / SSP-RK3 stage.
//
// Design (FP64 on B300 is the binding resource, HBM is not):
//  * k_prim: one thread per padded cell (interior + 3 ghost layers, boundary
//    conditions applied by index mapping). Newton temperature solve (Eq. 21)
//    on mixture-level polynomial coefficients, EOS (Eq. 7), sound speed,
//    total enthalpy and, when viscous, the Eq. 29 / Eq. 22 mixture transport.
//    Every per-cell quantity that the faces need is computed exactly once and
//    stored, so no FP64 work is repeated per face. Stage 1 fuses the CFL
//    max-reduction (warp shuffles, one atomic per block on ordered bits).
//  * k_grad: nodal 4th-order velocity derivatives (tangential terms of Eq. 3).
//  * k_face<D>: one thread per face of direction D. Roe-averaged face state,
//    the multicomponent eigensystem in the partial form of Sec. III.D.3 (per
//    field only its eigenvalue, its left row and its right column, all in
//    closed sparse form), LLF splitting (Eq. 14), two WENO5-JS reconstructions
//    per field normalised by one division per field, back-projection (Eq. 15), and the
//    viscous face flux. Writes G = F_hat - F_v per face.
//  * k_update: conservative difference (Eq. 13) and the SSP-RK3 combination
//    (Eq. 16), or the plain RHS.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace xf {

// ghost layers: 3 for the 6-cell stencils of WENO5 and CU6, 4 for WENO7
inline int ghosts(int weno) { return weno == 7 ? 4 : 3; }
constexpr int MAXN = 5;

struct Params {
  int dim, N, nv;
  int n[3];      // interior cells per axis (1 if inactive)
  int np[3];     // padded extents
  int go[3];     // ghost offset per axis (G or 0)
  int bc[3][2];
  long long cells, pcells;
  double inv_dx[3];
  // thermo, dimensionless (R_s / a_ref^2 pre-multiplied)
  double T_lo, span, inv_span;
  double tau0;            // -T_lo / span: tau = T inv_span + tau0
  double hsj[5];          // span / (j + 1): rh[s][j] = rcp[s][j] hsj[j]
  double r[MAXN];         // R_s / a_ref^2
  double rcp[MAXN][5];    // r_s cp_j: c_p,s = sum_j rcp[s][j] tau^j
  double rh[MAXN][5];     // r_s span cp_j/(j+1): h_s = rhoff_s + sum_j rh[s][j] tau^(j+1)
  double rhoff[MAXN];     // r_s h_off_s
  // the same for h_s - h_N (species s = 1..N-1): the face's heat flux by diffusion
  double rcpd[MAXN][5], rhd[MAXN][5], rhoffd[MAXN];
  double rdN[MAXN];        // r_s - r_N (s = 1..N-1): the face's phi_s - phi_N
  // transport
  double lnmu[MAXN][4], lnka[MAXN][4];
  double wA[MAXN][MAXN], wB[MAXN][MAXN];  // Wilke: A = (1+W_s/W_t)^-1/2 / sqrt 8, B = (W_t/W_s)^1/4
  double wAB[MAXN][MAXN], wABB[MAXN][MAXN];  // A B and A B^2
  double invW[MAXN], Wm[MAXN];  // 1/W_s and W_s (kg/mol)
  double fmu, fka, inv_lewis;
  int diffusion;                 // 0: D = kappa/(rho c_p Le); 1: mixture-averaged D_sm (Eq. 26)
  double dbin[MAXN][MAXN][4];    // ln(p D_st [Pa m^2/s]) cubic in ln T (Eq. 25, form of Eq. 29)
  double fdsm;                   // rho_ref a_ref^3 L_ref: 1/D*_st = p* fdsm exp(-ln(p D_st))
  // numerics
  double cfl, weno_eps, newton_rtol;
  double wenoe[4];   // epsilon terms of the reconstruction (rec_nd): 12 eps c_k
                     // (k < 3) and 12 eps for WENO5 / CU6, 240 eps c_k for WENO7
  double wenoe4[4];  // the same divided by 4: for data scaled by -1/2 (the
                     // reconstructions are homogeneous of degree one when eps
                     // scales with the square of the data, exactly so for a
                     // power-of-two factor)
  // the face kernel's fixed coefficients (kFaceCoef with the field pair's
  // division scale rec_scale at 14), read through dev like the run constants
  double kface[32];
  double kexp[8];    // kExpCoef (primitive recovery's exponentials)
  double klog[9];    // kLogCoef (primitive recovery's logarithm)
  int viscous, convective, newton_max;
  int weno;          // 5: WENO5-JS, 6: WENO-CU6
  int positivity;    // positivity-preserving blend of the convective flux (Eq. 17-20)
  double pos_eps;
  double hmin2_over_2dim;
  // This struct's copy in device memory, set by its owner (a solver handle, a
  // batch instance, the static scratch) before the first launch. The face
  // kernel and the primitive recovery read their FP64 coefficients from there:
  // an FP64 instruction that takes a kernel parameter or a literal as an
  // operand issues at about 84 % of the rate of one with register operands on
  // this GPU, and values loaded from memory land in registers.
  const Params* dev;
};

// Number of per-cell fields of Lay<dim, ns> (without the D_sm fields), for
// host code that sizes the field block from runtime (dim, N).
__host__ __device__ constexpr int lay_nq(int dim, int ns) {
  return (dim + 1 + ns) + dim + 5 + ns + 5 + 1 + 3 + 3 * dim + dim * dim;
}

// Padded per-cell field layout (SoA, stride pcells).
template <int DIM, int NS>
struct Lay {
  static constexpr int NV = DIM + 1 + NS;
  static constexpr int U = 0;           // conserved, BC applied
  static constexpr int UN = NV;         // velocity u_a
  static constexpr int P = UN + DIM;    // pressure
  static constexpr int C = P + 1;       // sound speed
  static constexpr int SR = C + 1;      // sqrt(rho)
  static constexpr int H = SR + 1;      // total enthalpy
  static constexpr int T = H + 1;       // temperature (K)
  static constexpr int Y = T + 1;       // Y_1..Y_N
  static constexpr int AC = Y + NS;     // mixture c_p coefficients A_0..A_4 (c_p = sum A_j tau^j)
  static constexpr int RM = AC + 5;     // mixture gas constant sum Y_s R_s
  static constexpr int MU = RM + 1;     // mixture viscosity
  static constexpr int KA = MU + 1;     // mixture conductivity
  static constexpr int DF = KA + 1;     // diffusivity
  // per axis a, for the face stencils of direction a: u_a/2, |u_a - c|/2 and
  // |u_a + c|/2 (each cell sits in six stencils per direction)
  static constexpr int HU = DF + 1;
  static constexpr int AM = HU + DIM;
  static constexpr int AP = AM + DIM;
  static constexpr int GU = AP + DIM;   // nodal d u_a / d x_b at GU + a*DIM + b
  static constexpr int NQ = GU + DIM * DIM;
  static constexpr int DS = NQ;         // D_sm of species 1..N, present (and
                                        // allocated) only with diffusion = 1
  static_assert(NQ == lay_nq(DIM, NS), "lay_nq must count the fields of Lay");
};

__device__ __forceinline__ double ld(const double* p) { return __ldg(p); }
// a coefficient read from the device copy of the parameters (Params::dev) into
// a register
__device__ __forceinline__ double rd(const double& x) { return __ldcg(&x); }

// 1/x by Newton-Raphson iteration for the reciprocal (M. J. Flynn, "On
// division by functional iteration", IEEE Trans. Computers C-19, 1970),
// started from the PTX approximation rcp.approx.ftz.f64: each step
// y <- y + y (1 - x y) doubles the number of correct bits, two steps reach
// double precision. For normal finite x (a subnormal x is flushed to zero,
// x = 0 or +-inf give NaN): the hot-path divisors (densities, heat
// capacities, WENO weight sums, mole-fraction sums) are all of that kind.
// xf_probe_rcp compares it with the correctly rounded 1.0 / x.
__device__ __forceinline__ double rcp_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}

// rcp_nr with the constant 1 of its iteration passed in a register
__device__ __forceinline__ double rcp_nr1(double x, double one) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, one);
  y = fma(y, e, y);
  e = fma(-x, y, one);
  return fma(y, e, y);
}

// 2^(j/64) for j = 0..63, each the double nearest the exact value (computed in
// exact decimal arithmetic and checked to lie within half an ulp of it).
static __device__ const double kExp2J64[64] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0,
    0x1.0874518759bc8p+0, 0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0,
    0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0, 0x1.172b83c7d517bp+0,
    0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0,
    0x1.2d285a6e4030bp+0, 0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0,
    0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0, 0x1.3dea64c123422p+0,
    0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0,
    0x1.56f4736b527dap+0, 0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0,
    0x1.6247eb03a5585p+0, 0x1.6623882552225p+0, 0x1.6a09e667f3bcdp+0,
    0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0,
    0x1.868d99b4492edp+0, 0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0,
    0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0, 0x1.9c49182a3f090p+0,
    0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0,
    0x1.bcc1e904bc1d2p+0, 0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0,
    0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0, 0x1.d5818dcfba487p+0,
    0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0,
    0x1.fa7c1819e90d8p+0,
};

// exp(x) for the transport fits by P. T. P. Tang's table-driven method
// ("Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM Trans. Math. Software 15, 1989):
// x = (64 m + j) ln2/64 + r with |r| <= ln2/128, and
// exp(x) = 2^m 2^(j/64) e^r, e^r = 1 + r + r^2 (1/2 + r/6 + r^2/24 + r^3/120)
// (the next Taylor term is below 4e-17 there). n = 64 m + j is rounded with
// the 1.5 2^52 shift, r is formed with ln2/64 split into a leading double and
// its remainder, 2^(j/64) comes from the table and 2^m is added to the
// exponent on the integer pipe: 10 FP64 instructions. Within about one ulp
// of exp (xf_probe_exp). |x| > 700 (outside the fits' range; the test runs on
// the bit pattern) takes exp.
// Its constants, in the order exp_k takes them: 64/ln 2, the 1.5 2^52 shift,
// -(ln 2/64) split into a leading double and its remainder, and the Taylor
// coefficients 1/120, 1/24, 1/6, 1/2.
#define XF_EXP_COEF                                                          \
  0x1.71547652b82fep+6, 6755399441055744.0, -0x1.62e42fefa39efp-7, -0x1.abc9e3b39803fp-62, \
      1.0 / 120.0, 1.0 / 24.0, 1.0 / 6.0, 0.5
constexpr double kExpCoef[8] = {XF_EXP_COEF};
// K = kExpCoef, as literals (exp_t) or loaded into registers (primitive
// recovery, from the device copy of the parameters)
__device__ __forceinline__ double exp_k(double x, const double* K) {
  if (!((__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL) <= 0x4085E00000000000LL))  // |x| <= 700
    return exp(x);
  const double t = fma(x, K[0], K[1]);
  const long long n = __double_as_longlong(t) - __double_as_longlong(6755399441055744.0);
  const double kd = t - K[1];
  const double r = fma(kd, K[3], fma(kd, K[2], x));
  const double q = fma(fma(fma(K[4], r, K[5]), r, K[6]), r, K[7]);
  const double er1 = fma(r * r, q, r);               // e^r - 1
  const double T = __ldg(kExp2J64 + (n & 63));
  const double e = fma(T, er1, T);
  return __longlong_as_double(__double_as_longlong(e) +
                              (long long)((unsigned long long)(n >> 6) << 52));
}
__device__ __forceinline__ double exp_t(double x) {
  const double K[8] = {XF_EXP_COEF};
  return exp_k(x, K);
}

// 1/F at the nodes F = 1 + j/128, j = 0..128, each the double nearest the
// exact value; ln F split as hi + lo, hi the multiple of 2^-43 nearest ln F
// and lo the double nearest the rest (computed in 300-bit arithmetic and
// checked to lie within half an ulp).
static __device__ const double kInvF128[129] = {
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
    0x1.0204081020408p-1, 0x1.0101010101010p-1, 0x1.0000000000000p-1,
};
static __device__ const double kLnF128Hi[129] = {
    0x0.0p+0, 0x1.fe02a6b100000p-8, 0x1.fc0a8b0fc0000p-7,
    0x1.7b91b07d58000p-6, 0x1.f829b0e780000p-6, 0x1.39e87b9fec000p-5,
    0x1.77458f632c000p-5, 0x1.b42dd71198000p-5, 0x1.f0a30c0118000p-5,
    0x1.16536eea38000p-4, 0x1.341d7961be000p-4, 0x1.51b073f062000p-4,
    0x1.6f0d28ae56000p-4, 0x1.8c345d631a000p-4, 0x1.a926d3a4ae000p-4,
    0x1.c5e548f5bc000p-4, 0x1.e27076e2b0000p-4, 0x1.fec9131dbe000p-4,
    0x1.0d77e7cd09000p-3, 0x1.1b72ad52f6000p-3, 0x1.29552f81ff000p-3,
    0x1.371fc201e9000p-3, 0x1.44d2b6ccb8000p-3, 0x1.526e5e3a1b000p-3,
    0x1.5ff3070a79000p-3, 0x1.6d60fe719d000p-3, 0x1.7ab890210e000p-3,
    0x1.87fa06520d000p-3, 0x1.9525a9cf45000p-3, 0x1.a23bc1fe2b000p-3,
    0x1.af3c94e80c000p-3, 0x1.bc286742d9000p-3, 0x1.c8ff7c79aa000p-3,
    0x1.d5c216b4fc000p-3, 0x1.e27076e2af000p-3, 0x1.ef0adcbdc6000p-3,
    0x1.fb9186d5e4000p-3, 0x1.0402594b4d000p-2, 0x1.0a324e2739000p-2,
    0x1.1058bf9ae4800p-2, 0x1.1675cababa800p-2, 0x1.1c898c1699800p-2,
    0x1.22941fbcf7800p-2, 0x1.2895a13de8800p-2, 0x1.2e8e2bae12000p-2,
    0x1.347dd9a988000p-2, 0x1.3a64c55694800p-2, 0x1.404308686a800p-2,
    0x1.4618bc21c6000p-2, 0x1.4be5f95777800p-2, 0x1.51aad872df800p-2,
    0x1.5767717455800p-2, 0x1.5d1bdbf580800p-2, 0x1.62c82f2b9c800p-2,
    0x1.686c81e9b1800p-2, 0x1.6e08eaa2ba000p-2, 0x1.739d7f6bbd000p-2,
    0x1.792a55fdd4800p-2, 0x1.7eaf83b82b000p-2, 0x1.842d1da1e8800p-2,
    0x1.89a3386c14000p-2, 0x1.8f11e87366000p-2, 0x1.947941c211800p-2,
    0x1.99d958117e000p-2, 0x1.9f323ecbf9800p-2, 0x1.a484090e5b800p-2,
    0x1.a9cec9a9a0800p-2, 0x1.af12932477800p-2, 0x1.b44f77bcc9000p-2,
    0x1.b985896931000p-2, 0x1.beb4d9da71800p-2, 0x1.c3dd7a7cdb000p-2,
    0x1.c8ff7c79a9800p-2, 0x1.ce1af0b85f000p-2, 0x1.d32fe7e00e800p-2,
    0x1.d83e7258a3000p-2, 0x1.dd46a04c1c800p-2, 0x1.e24881a7c7000p-2,
    0x1.e744261d68800p-2, 0x1.ec399d2469000p-2, 0x1.f128f5faf0800p-2,
    0x1.f6123fa702800p-2, 0x1.faf588f78f000p-2, 0x1.ffd2e0857f800p-2,
    0x1.02552a5a5d000p-1, 0x1.04bdf9da92800p-1, 0x1.0723e5c1ce000p-1,
    0x1.0986f4f573400p-1, 0x1.0be72e4252c00p-1, 0x1.0e44985d1cc00p-1,
    0x1.109f39e2d4c00p-1, 0x1.12f719593f000p-1, 0x1.154c3d2f4d400p-1,
    0x1.179eabbd89800p-1, 0x1.19ee6b467c800p-1, 0x1.1c3b81f713c00p-1,
    0x1.1e85f5e704000p-1, 0x1.20cdcd192ac00p-1, 0x1.23130d7bec000p-1,
    0x1.2555bce98f800p-1, 0x1.2795e1289b000p-1, 0x1.29d37fec2b000p-1,
    0x1.2c0e9ed449000p-1, 0x1.2e47436e40400p-1, 0x1.307d7334f1000p-1,
    0x1.32b1339121c00p-1, 0x1.34e289d9ce000p-1, 0x1.37117b5474800p-1,
    0x1.393e0d3562c00p-1, 0x1.3b68449fffc00p-1, 0x1.3d9026a715800p-1,
    0x1.3fb5b84d17000p-1, 0x1.41d8fe8467400p-1, 0x1.43f9fe2f9d000p-1,
    0x1.4618bc21c6000p-1, 0x1.48353d1ea8800p-1, 0x1.4a4f85db04000p-1,
    0x1.4c679afccf000p-1, 0x1.4e7d811b75c00p-1, 0x1.50913cc016800p-1,
    0x1.52a2d265bc400p-1, 0x1.54b2467999400p-1, 0x1.56bf9d5b3f400p-1,
    0x1.58cadb5cd7800p-1, 0x1.5ad404c35a000p-1, 0x1.5cdb1dc6c1800p-1,
    0x1.5ee02a9241800p-1, 0x1.60e32f4478800p-1, 0x1.62e42fefa3800p-1,
};
static __device__ const double kLnF128Lo[129] = {
    0x0.0p+0, 0x1.9e23f0dda40e4p-46, 0x1.f1e7cf6d3a69cp-50,
    0x1.88d5493faa639p-45, 0x1.980267c7e09e4p-45, -0x1.502b7f526feaap-48,
    0x1.cfc4634f2a1eep-45, -0x1.c827ae5d6704cp-46, -0x1.d599e83368e91p-45,
    -0x1.47c5e768fa309p-46, -0x1.c5edaccf913dfp-45, -0x1.f025b61c65e57p-46,
    0x1.69737c93373dap-45, -0x1.37c294d2f5668p-46, -0x1.53935e85baac8p-45,
    0x1.d0c57585fbe06p-46, -0x1.a342c2af0003cp-45, 0x1.575545ca333f2p-45,
    -0x1.a699688e85bf4p-47, 0x1.e80a41811a396p-45, 0x1.48d301771c408p-45,
    -0x1.178864d27543ap-48, -0x1.70cc16135783cp-46, 0x1.0de8b90075b8fp-45,
    0x1.e9e439f105039p-46, 0x1.0e46aa3b2e266p-46, -0x1.bdb9072534a58p-45,
    -0x1.bbdbf7fdbfa09p-45, 0x1.ad1d904c1d4e3p-45, 0x1.58c64dc46c1eap-45,
    -0x1.a4e633fcd9066p-52, -0x1.94eb0318bb78fp-46, -0x1.7794f689f8434p-45,
    -0x1.1ba91bbca681bp-45, 0x1.72f4f543fff10p-46, -0x1.b26b79c86af24p-45,
    -0x1.d572aab993c87p-47, 0x1.036b89ef42d7fp-48, 0x1.c6bee7ef4030ep-47,
    0x1.6a8c4fd055a66p-45, -0x1.f1fc63382a8f0p-46, 0x1.fafbc68e75404p-46,
    0x1.65a242853da76p-46, -0x1.5ca14b6cfb03fp-46, -0x1.67b1e99b72bd8p-45,
    -0x1.5594dd4c58092p-45, -0x1.0b1c686519460p-45, -0x1.c42f3ed820b3ap-50,
    -0x1.3d82f484c84ccp-46, 0x1.41b6993293ee0p-47, 0x1.684e49eb067d5p-49,
    0x1.362a4d5b6506dp-45, 0x1.ca508d8e0f720p-46, -0x1.ab42428375680p-48,
    -0x1.a89ddea0f7f59p-45, 0x1.e38c139318d71p-46, 0x1.a7389314feb50p-52,
    -0x1.760fa896e0161p-48, -0x1.e4da62d0c25adp-49, 0x1.8ba49d8a32f09p-45,
    0x1.2d5ad38c40882p-45, 0x1.63bf0bb4eab4cp-45, -0x1.0545b322eb82fp-46,
    0x1.1597525dd88f0p-47, 0x1.2fcada35d9bd0p-48, 0x1.8515fe535b876p-45,
    0x1.2635213fd4bc9p-48, 0x1.ac44ce1128577p-48, -0x1.3ae68224aa2cep-47,
    0x1.f6b31f629f11ep-47, 0x1.bdfbc30e9bd5ep-45, -0x1.5946261f5a42bp-45,
    0x1.10d612ec0f798p-45, 0x1.f5bdbe95e5568p-45, 0x1.eab0ef6465f5fp-45,
    -0x1.835f5d48ba26dp-47, -0x1.afa08cecadb17p-45, -0x1.ecf1a1385d356p-45,
    -0x1.e0720972430d1p-48, -0x1.9ff45188d6065p-45, -0x1.134ca37c4eecep-46,
    0x1.58c28ad8796dap-47, 0x1.8f6cd7d9f2754p-45, -0x1.b3d53417e4d9cp-45,
    0x1.fd8d38d2bafddp-46, -0x1.2d9a033eff74ep-45, -0x1.7f6350d38edddp-46,
    0x1.20b91fda94ff4p-45, -0x1.7d49676844cc2p-45, 0x1.17edd5cbbd2d3p-46,
    0x1.2dfbc7d93616fp-46, -0x1.0eb3fb7398e0cp-47, 0x1.e9a98f33a3966p-45,
    0x1.a0bfc60e6fa08p-45, 0x1.6ecc5cbdd7782p-45, 0x1.25e4a7c766fdep-48,
    0x1.a07bd8b34be7cp-46, -0x1.24d95f85e1148p-46, -0x1.7afa4392f1ba7p-46,
    -0x1.a61fde292977ep-48, 0x1.1aeb783f3db97p-45, 0x1.1590b9ad974bap-46,
    -0x1.74468563ce45dp-45, -0x1.97bfabde796dep-45, 0x1.7c3f6b2143eadp-46,
    0x1.71320556b67b2p-45, 0x1.d316eb92d885dp-45, -0x1.28e88bf6deec9p-47,
    -0x1.e6563bbd9fc92p-45, 0x1.157c76f60c2cap-48, -0x1.055bfbd9c2f53p-45,
    -0x1.7b4962c55f46bp-46, -0x1.519b9b433d0bap-45, -0x1.98858d84649f1p-45,
    -0x1.3d82f484c84ccp-45, 0x1.bee7abd176604p-46, -0x1.44fdd840b8591p-45,
    -0x1.c64e971322ce8p-45, -0x1.3d8d3d9ea6e9fp-47, 0x1.ad2f2ce96c2d6p-47,
    0x1.aaee77c8af15bp-45, 0x1.2f522a851687bp-46, -0x1.9afb8e77a3270p-47,
    0x1.893092f25d931p-45, -0x1.a609acaab41fcp-46, -0x1.36e612387451fp-46,
    -0x1.8a8f29f6a02dcp-45, 0x1.b194f912b416ap-46, 0x1.ef35793c76730p-45,
};

// ln x for the transport fits' ln T by P. T. P. Tang's table-driven method
// ("Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM Trans. Math. Software 16, 1990): x = 2^m y
// with y in [1, 2); F = 1 + j/128 is the node nearest y, so f = y - F is exact
// (|f| <= 1/256); u = f/F with 1/F from the table; and
// ln x = (m ln2_hi + lnF_hi) + (m ln2_lo + lnF_lo + ln(1 + u)): both hi parts
// are multiples of 2^-43, so their sum is exact for any exponent m (no
// cancellation error near x = 1), and ln(1 + u) = u + u^2 q(u) with
// q = -1/2 + u/3 - ... - u^6/8 (the next term is below 3e-21 for
// |u| <= 1/256). 14 FP64 arithmetic instructions and one conversion, against
// 28 for CUDA's log; within one ulp of the correctly rounded value
// (xf_probe_log). x outside the positive normal doubles takes log.
// Its constants, in the order log_k takes them: -1/8, 1/7, -1/6, 1/5, -1/4,
// 1/3, -1/2 and ln 2 split as ln2_hi (a multiple of 2^-43) + ln2_lo.
#define XF_LOG_COEF                                                               \
  -1.0 / 8.0, 1.0 / 7.0, -1.0 / 6.0, 0.2, -0.25, 1.0 / 3.0, -0.5, 0x1.62e42fefa3800p-1, \
      0x1.ef35793c76730p-45
constexpr double kLogCoef[9] = {XF_LOG_COEF};
// K = kLogCoef, as literals (log_t) or loaded into registers (primitive
// recovery, from the device copy of the parameters)
__device__ __forceinline__ double log_k(double x, const double* K) {
  const long long b = __double_as_longlong(x);
  // positive normal x: the bit pattern in [2^52, 0x7FF0000000000000)
  if (!((unsigned long long)(b - 0x0010000000000000LL) < 0x7FE0000000000000ULL)) return log(x);
  const double md = (double)((int)(b >> 52) - 1023);
  const long long mant = b & 0x000FFFFFFFFFFFFFLL;
  const int j = (int)((mant + (1LL << 44)) >> 45);   // the nearest node, 0..128
  const double y = __longlong_as_double(mant | 0x3FF0000000000000LL);
  const double F = __longlong_as_double(0x3FF0000000000000LL + ((long long)j << 45));
  const double u = (y - F) * __ldg(kInvF128 + j);
  double q = fma(K[0], u, K[1]);
#pragma unroll
  for (int k = 2; k < 7; ++k) q = fma(q, u, K[k]);
  const double hi = fma(md, K[7], __ldg(kLnF128Hi + j));   // exact
  const double lo = fma(md, K[8], __ldg(kLnF128Lo + j)) + fma(u * u, q, u);
  return hi + lo;
}
__device__ __forceinline__ double log_t(double x) {
  const double K[9] = {XF_LOG_COEF};
  return log_k(x, K);
}

// max of two non-negative doubles through their ordered bit patterns (integer
// pipe; the FP64 pipe is the scarce unit)
__device__ __forceinline__ double pmax(double a, double b) {
  long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
}

// Boundary mapping of one axis (mirrors XF_BC_*): returns the interior index
// that feeds padded index i and sets *flip for a symmetric mirror.
__device__ __forceinline__ int map_axis(int i, int n, int lo, int hi, bool* flip) {
  *flip = false;
  if (i >= 0 && i < n) return i;
  int bc = i < 0 ? lo : hi;
  if (bc == 1) return i < 0 ? i + n : i - n;
  if (bc == 2) { *flip = true; return i < 0 ? -1 - i : 2 * n - 1 - i; }
  return i < 0 ? 0 : n - 1;
}

// ------------------------------------------------------------ thermo ------
// c_p,s(T) and h_s(T) of one species at a clamped tau, with the enthalpy
// continued linearly (slope c_p at the end point) outside [T_lo, T_hi].
struct TauPt {
  double tc;   // clamped tau
  double ext;  // span * (tau - tc)
  bool in;     // tau in [0, 1] (then tc = tau, ext = 0)
};
__device__ __forceinline__ TauPt tau_pt(const Params& p, double tau) {
  TauPt r;
  // the range test on the bit pattern (non-negative doubles order as
  // integers) keeps the common in-range case off the FP64 pipe
  const long long b = __double_as_longlong(tau);
  r.in = b >= 0 && b <= 0x3FF0000000000000LL;
  if (r.in) {
    r.tc = tau;
    r.ext = 0.0;
  } else {
    r.tc = fmin(fmax(tau, 0.0), 1.0);
    r.ext = p.span * (tau - r.tc);
  }
  return r;
}
__device__ __forceinline__ TauPt tau_of(const Params& p, double T) {
  return tau_pt(p, fma(T, p.inv_span, p.tau0));
}
__device__ __forceinline__ double cp_s(const Params& p, int s, double tc) {
  const double* a = p.rcp[s];
  return fma(fma(fma(fma(a[4], tc, a[3]), tc, a[2]), tc, a[1]), tc, a[0]);
}
__device__ __forceinline__ double h_s(const Params& p, int s, const TauPt& t, double cps) {
  const double* a = p.rh[s];
  double poly = fma(fma(fma(fma(a[4], t.tc, a[3]), t.tc, a[2]), t.tc, a[1]), t.tc, a[0]);
  return fma(poly, t.tc, p.rhoff[s]) + cps * t.ext;
}

// h_s alone: the c_p term of the linear continuation is evaluated only when T
// lies outside [T_lo, T_hi]; inside (ext = 0), the result is the same bits.
__device__ __forceinline__ double h_s_in(const Params& p, int s, const TauPt& t) {
  const double* a = p.rh[s];
  const double poly = fma(fma(fma(fma(a[4], t.tc, a[3]), t.tc, a[2]), t.tc, a[1]), t.tc, a[0]);
  const double h = fma(poly, t.tc, p.rhoff[s]);
  return t.in ? h : fma(cp_s(p, s, t.tc), t.ext, h);
}

// h_s_in with the coefficients read from the device copy of the parameters
// (register operands; the same arithmetic)
__device__ __forceinline__ double h_s_dev(const Params& p, int s, const TauPt& t) {
  const double* a = p.dev->rh[s];
  const double poly = fma(fma(fma(fma(__ldcg(a + 4), t.tc, __ldcg(a + 3)), t.tc, __ldcg(a + 2)),
                              t.tc, __ldcg(a + 1)),
                          t.tc, __ldcg(a + 0));
  const double h = fma(poly, t.tc, __ldcg(p.dev->rhoff + s));
  return t.in ? h : fma(cp_s(p, s, t.tc), t.ext, h);
}

// c_p,s - c_p,N at the clamped tau, from the parameters' device copy
__device__ __forceinline__ double cpd_s_dev(const Params& p, int s, double tc) {
  const double* c = p.dev->rcpd[s];
  return fma(fma(fma(fma(__ldcg(c + 4), tc, __ldcg(c + 3)), tc, __ldcg(c + 2)), tc,
                 __ldcg(c + 1)),
             tc, __ldcg(c + 0));
}

// h_s - h_N with the coefficients' differences from the parameters' device
// copy (register operands; the linear continuation as in h_s_in)
__device__ __forceinline__ double hd_s_dev(const Params& p, int s, const TauPt& t) {
  const double* a = p.dev->rhd[s];
  const double poly = fma(fma(fma(fma(__ldcg(a + 4), t.tc, __ldcg(a + 3)), t.tc, __ldcg(a + 2)),
                              t.tc, __ldcg(a + 1)),
                          t.tc, __ldcg(a + 0));
  const double h = fma(poly, t.tc, __ldcg(p.dev->rhoffd + s));
  if (t.in) return h;
  const double* c = p.rcpd[s];
  const double cpd = fma(fma(fma(fma(c[4], t.tc, c[3]), t.tc, c[2]), t.tc, c[1]), t.tc, c[0]);
  return fma(cpd, t.ext, h);
}

// ------------------------------------------------------------ status ------
__device__ __forceinline__ void raise(uint32_t* flags, uint32_t bits) {
  if (bits) atomicOr(flags, bits);
}

// ================================================================ k_prim ===
// One thread per padded cell. Reads conserved U (interior, BC by mapping),
// writes the padded per-cell fields. Stage-1 launches also reduce the CFL
// maxima over interior cells into red[0] (sum_d (|u_d|+c)/dx_d) and red[1]
// (viscous diffusivity), as ordered bit patterns of non-negative doubles.
// Per-cell body of the primitive recovery (shared by the plain kernel and the
// batched persistent kernel, so both run the same arithmetic). t is the padded
// cell index (t < pcells); s_cfl / s_nu receive this cell's CFL terms.
template <int DIM, int NS>
__device__ __forceinline__ void prim_cell(const Params& p, long long t, const double* __restrict__ U,
                                          const double* __restrict__ Tin, double* __restrict__ Tout,
                                          double* __restrict__ Q, uint32_t* __restrict__ flags,
                                          int do_cfl, double& s_cfl, double& s_nu) {
  using L = Lay<DIM, NS>;
  constexpr int NV = L::NV;
  const long long PC = p.pcells;
  {
    const int ip = (int)(t % p.np[0]);
    const int jp = (int)((t / p.np[0]) % p.np[1]);
    const int kp = (int)(t / ((long long)p.np[0] * p.np[1]));
    const int i = ip - p.go[0], j = jp - p.go[1], k = kp - p.go[2];
    bool f0 = false, f1 = false, f2 = false;
    const int si = map_axis(i, p.n[0], p.bc[0][0], p.bc[0][1], &f0);
    const int sj = DIM > 1 ? map_axis(j, p.n[1], p.bc[1][0], p.bc[1][1], &f1) : 0;
    const int sk = DIM > 2 ? map_axis(k, p.n[2], p.bc[2][0], p.bc[2][1], &f2) : 0;
    const bool interior = (si == i) && (sj == j) && (sk == k);
    const long long src = ((long long)sk * p.n[1] + sj) * p.n[0] + si;
    const long long C = p.cells;
    double u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = ld(U + v * C + src);
    if (f0) u[1] = -u[1];
    if (DIM > 1 && f1) u[2] = -u[2];
    if (DIM > 2 && f2) u[3] = -u[3];
    uint32_t st = 0;
    bool finite = true;
#pragma unroll
    for (int v = 0; v < NV; ++v) finite = finite && isfinite(u[v]);
    // the FP64 coefficients below come from the parameters' device copy
    // (register operands, Params::dev)
    const Params& pd = *p.dev;
    const double one = rd(pd.kface[13]), half = rd(pd.kexp[7]);
    const double rho = u[0];
    const double irho = rcp_nr1(rho, one);
    double vel[DIM], ke = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) { vel[a] = u[1 + a] * irho; ke = fma(vel[a], vel[a], ke); }
    const double E = u[DIM + 1];
    double Y[NS], ysum = 0.0;
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) { Y[s] = u[DIM + 2 + s] * irho; ysum += Y[s]; }
    Y[NS - 1] = one - ysum;
    const double e = fma(E, irho, -(half * ke));
    // mixture polynomial coefficients: c_p(tau) = sum A_j tau^j,
    // h(tau) = B + sum Ah_j tau^(j+1) with Ah_j = A_j span/(j+1), R = Rm
    double A[5], Ah[5], Rm = 0.0, B = 0.0;
#pragma unroll
    for (int jj = 0; jj < 5; ++jj) A[jj] = 0.0;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      Rm = fma(Y[s], rd(pd.r[s]), Rm);
      B = fma(Y[s], rd(pd.rhoff[s]), B);
#pragma unroll
      for (int jj = 0; jj < 5; ++jj) A[jj] = fma(Y[s], rd(pd.rcp[s][jj]), A[jj]);
    }
#pragma unroll
    for (int jj = 0; jj < 5; ++jj) Ah[jj] = A[jj] * rd(pd.hsj[jj]);
    // Newton (Eq. 21): T <- T + (e - e(T)) / c_v(T), stop at |dT| <= rtol T;
    // a non-positive iterate is replaced by half the previous one
    double T = ld(Tin + src);
    const double isp = rd(pd.inv_span), tau0 = rd(pd.tau0), rtol = rd(pd.newton_rtol);
    bool conv = false;
    for (int it = 0; it < p.newton_max; ++it) {
      const TauPt tp = tau_pt(p, fma(T, isp, tau0));
      const double cpm = fma(fma(fma(fma(A[4], tp.tc, A[3]), tp.tc, A[2]), tp.tc, A[1]), tp.tc, A[0]);
      const double hp = fma(fma(fma(fma(fma(Ah[4], tp.tc, Ah[3]), tp.tc, Ah[2]), tp.tc, Ah[1]), tp.tc, Ah[0]), tp.tc, B);
      const double eT = (tp.in ? hp : fma(cpm, tp.ext, hp)) - Rm * T;
      double Tn = fma(e - eT, rcp_nr1(cpm - Rm, one), T);
      if (!(Tn > 0.0)) Tn = half * T;
      conv = fabs(Tn - T) <= rtol * Tn;
      T = Tn;
      if (conv) break;
    }
    if (!conv) st |= 2u;
    const TauPt tp = tau_pt(p, fma(T, isp, tau0));
    const double cpm = fma(fma(fma(fma(A[4], tp.tc, A[3]), tp.tc, A[2]), tp.tc, A[1]), tp.tc, A[0]);
    const double cvm = cpm - Rm;
    const double RT = Rm * T;
    const double pr = rho * RT;
    const double icvm = rcp_nr1(cvm, one);
    const double c2 = cpm * RT * icvm;
    const double c = sqrt(c2);
    const double H = (E + pr) * irho;
    if (!finite || !(rho > 0.0) || !(pr > 0.0) || !(T > 0.0)) st |= 1u;
    double* q = Q + t;
#pragma unroll
    for (int v = 0; v < NV; ++v) q[(L::U + v) * PC] = u[v];
#pragma unroll
    for (int a = 0; a < DIM; ++a) q[(L::UN + a) * PC] = vel[a];
    q[L::P * PC] = pr;
    q[L::C * PC] = c;
    q[L::SR * PC] = sqrt(rho);
    q[L::H * PC] = H;
    q[L::T * PC] = T;
#pragma unroll
    for (int s = 0; s < NS; ++s) q[(L::Y + s) * PC] = Y[s];
#pragma unroll
    for (int jj = 0; jj < 5; ++jj) q[(L::AC + jj) * PC] = A[jj];
    q[L::RM * PC] = Rm;
    {
      const double hc = half * c;
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const double hu = half * vel[a];
        q[(L::HU + a) * PC] = hu;
        q[(L::AM + a) * PC] = fabs(hu - hc);
        q[(L::AP + a) * PC] = fabs(hu + hc);
      }
    }
    double mu = 0.0, ka = 0.0, Dd = 0.0;
    if (p.viscous) {
      // Eq. 29 fits; sqrt(mu_s) = exp(ln mu_s / 2) feeds the Wilke ratios (Eq. 22)
      double KL[9];
#pragma unroll
      for (int j = 0; j < 9; ++j) KL[j] = rd(pd.klog[j]);
      const double lnT = log_k(T, KL);
      double KX[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) KX[j] = rd(pd.kexp[j]);
      double smu[NS], ska[NS], ismu[NS], iska[NS], X[NS], xs = 0.0;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const double* fm = pd.lnmu[s];
        const double* fk = pd.lnka[s];
        const double lm = fma(fma(fma(rd(fm[3]), lnT, rd(fm[2])), lnT, rd(fm[1])), lnT, rd(fm[0]));
        const double lk = fma(fma(fma(rd(fk[3]), lnT, rd(fk[2])), lnT, rd(fk[1])), lnT, rd(fk[0]));
        smu[s] = exp_k(half * lm, KX);
        ska[s] = exp_k(half * lk, KX);
        X[s] = Y[s] * rd(pd.invW[s]);
        xs += X[s];
      }
      // the 2N reciprocals 1/sqrt(mu_s), 1/sqrt(kappa_s) from one division
      // (running products: 1/v_k = (prod_{j<k} v_j) / (prod_{j<=k} v_j))
      {
        double pre[2 * NS];
        pre[0] = smu[0];
#pragma unroll
        for (int k = 1; k < 2 * NS; ++k) pre[k] = pre[k - 1] * (k < NS ? smu[k] : ska[k - NS]);
        double inv = rcp_nr1(pre[2 * NS - 1], one);
#pragma unroll
        for (int k = 2 * NS - 1; k > 0; --k) {
          const double v = k < NS ? smu[k] : ska[k - NS];
          const double r = inv * pre[k - 1];
          if (k < NS) ismu[k] = r; else iska[k - NS] = r;
          inv *= v;
        }
        ismu[0] = inv;
      }
      const double ixs = rcp_nr1(xs, one);
      // Wilke denominators sum_t X_t A_st (1 + r_st B_st)^2 with r_st = (a_s/a_t)^(1/2),
      // expanded: S0_s + 2 sqrt(a_s) S1_s + a_s S2_s, where S0_s = sum_t X_t A_st,
      // S1_s = sum_t X_t a_t^(-1/2) A_st B_st, S2_s = sum_t X_t a_t^(-1) A_st B_st^2
      // (all terms positive); S0 is shared by mu and kappa.
      double xm1[NS], xm2[NS], xk1[NS], xk2[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        X[s] *= ixs;
        xm1[s] = X[s] * ismu[s];
        xm2[s] = xm1[s] * ismu[s];
        xk1[s] = X[s] * iska[s];
        xk2[s] = xk1[s] * iska[s];
      }
      // The diagonal t = s contributes exactly X_s (Phi_ss = 1: A_ss = 1/4,
      // B_ss = 1), added once instead of through the five sums.
      double dm[NS], dk[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        double s0 = 0.0, m1 = 0.0, m2 = 0.0, k1 = 0.0, k2 = 0.0;
#pragma unroll
        for (int tt = 0; tt < NS; ++tt) {
          if (tt == s) continue;
          const double wab = rd(pd.wAB[s][tt]), wabb = rd(pd.wABB[s][tt]);
          s0 = fma(X[tt], rd(pd.wA[s][tt]), s0);
          m1 = fma(xm1[tt], wab, m1);
          m2 = fma(xm2[tt], wabb, m2);
          k1 = fma(xk1[tt], wab, k1);
          k2 = fma(xk2[tt], wabb, k2);
        }
        s0 += X[s];
        dm[s] = fma(smu[s] * smu[s], m2, fma(smu[s] + smu[s], m1, s0));
        dk[s] = fma(ska[s] * ska[s], k2, fma(ska[s] + ska[s], k1, s0));
      }
      // the 2N Wilke denominators inverted with one division, as above
      {
        double pre[2 * NS];
        pre[0] = dm[0];
#pragma unroll
        for (int k = 1; k < 2 * NS; ++k) pre[k] = pre[k - 1] * (k < NS ? dm[k] : dk[k - NS]);
        double inv = rcp_nr1(pre[2 * NS - 1], one);
        double idm[NS], idk[NS];
#pragma unroll
        for (int k = 2 * NS - 1; k > 0; --k) {
          const double v = k < NS ? dm[k] : dk[k - NS];
          const double r = inv * pre[k - 1];
          if (k < NS) idm[k] = r; else idk[k - NS] = r;
          inv *= v;
        }
        idm[0] = inv;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          mu = fma(X[s] * (smu[s] * smu[s]), idm[s], mu);
          ka = fma(X[s] * (ska[s] * ska[s]), idk[s], ka);
        }
      }
      mu *= rd(pd.fmu);
      ka *= rd(pd.fka);
      Dd = ka * rd(pd.inv_lewis) * rcp_nr1(rho * cpm, one);
      q[L::MU * PC] = mu;
      q[L::KA * PC] = ka;
      q[L::DF * PC] = Dd;
      if (p.diffusion == 1) {
        // Eq. 25-26: D_sm = sum_{t!=s} X~_t W_t / (W~ sum_{t!=s} X~_t / D_st) with
        // X~ = (max(X, 0) + 1e-12) normalised and W~ = sum_t X~_t W_t; the fits
        // give 1/D*_st = p* fdsm exp(-l_st(ln T)), one exp per pair.
        double Xt[NS], xts = 0.0;
#pragma unroll
        for (int s = 0; s < NS; ++s) { Xt[s] = fmax(X[s], 0.0) + 1e-12; xts += Xt[s]; }
        const double ixts = rcp_nr1(xts, one);
        // the sums of products are written as fused multiply-adds: the
        // batched kernel compiles this body too and must give the same bits
        double Wt = 0.0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          Xt[s] *= ixts;
          Wt = fma(Xt[s], rd(pd.Wm[s]), Wt);
        }
        double den[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) den[s] = 0.0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
#pragma unroll
          for (int tt = s + 1; tt < NS; ++tt) {
            const double* b = pd.dbin[s][tt];
            const double l = fma(fma(fma(rd(b[3]), lnT, rd(b[2])), lnT, rd(b[1])), lnT, rd(b[0]));
            const double iD = exp_k(-l, KX);
            den[s] = fma(Xt[tt], iD, den[s]);
            den[tt] = fma(Xt[s], iD, den[tt]);
          }
        }
        const double sc = rcp_nr1(Wt * pr * rd(pd.fdsm), one);
        double Dmax = 0.0;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          double num = 0.0;
#pragma unroll
          for (int tt = 0; tt < NS; ++tt)
            if (tt != s) num = fma(Xt[tt], rd(pd.Wm[tt]), num);
          const double Ds = num * sc * rcp_nr1(den[s], one);
          q[(L::DS + s) * PC] = Ds;
          Dmax = fmax(Dmax, Ds);
        }
        Dd = Dmax;  // the CFL limit takes the largest species diffusivity
      }
    }
    if (interior) {
      Tout[src] = T;
      if (do_cfl) {
        double sc = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) sc = fma(fabs(vel[a]) + c, p.inv_dx[a], sc);
        s_cfl = sc;
        if (p.viscous) {
          const double nu1 = (4.0 / 3.0) * mu * irho;
          const double nu2 = ka * irho * icvm;
          s_nu = pmax(pmax(nu1, nu2), Dd);
        }
      }
    }
    raise(flags, st);
    }
}

// Block-wide max of (a, b) over ordered bit patterns, one atomicMax per block.
__device__ __forceinline__ void block_max2(double s_cfl, double s_nu, unsigned long long* red) {
  unsigned long long a = (unsigned long long)__double_as_longlong(s_cfl);
  unsigned long long b = (unsigned long long)__double_as_longlong(s_nu);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long a2 = __shfl_xor_sync(0xffffffffu, a, o);
    const unsigned long long b2 = __shfl_xor_sync(0xffffffffu, b, o);
    a = a2 > a ? a2 : a;
    b = b2 > b ? b2 : b;
  }
  __shared__ unsigned long long sa[32], sb[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      a = sa[k] > a ? sa[k] : a;
      b = sb[k] > b ? sb[k] : b;
    }
    atomicMax(red + 0, a);
    atomicMax(red + 1, b);
  }
}

// Interior cells [c0, c1) (0 <= c0 <= c1 <= cells; the whole grid, or one
// slab of planes of the slowest axis), each written at its padded position.
// The ghost layers are filled afterwards by k_ghost. Two blocks per SM (at
// most 128 registers, a few spilled) ran 4.7 % faster than one block with
// the 166 registers the compiler takes otherwise.
template <int DIM, int NS>
__global__ void __launch_bounds__(256, 2)
k_prim(const __grid_constant__ Params p, const double* __restrict__ U,
       const double* __restrict__ Tin, double* __restrict__ Tout,
       double* __restrict__ Q, uint32_t* __restrict__ flags,
       unsigned long long* __restrict__ red, int do_cfl, long long c0, long long c1) {
  const long long c = c0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double s_cfl = 0.0, s_nu = 0.0;
  if (c < c1) {
    const unsigned cu = (unsigned)c, n0 = (unsigned)p.n[0], n1 = (unsigned)p.n[1];
    const unsigned q = cu / n0;
    const long long i = cu - q * n0, j = q % n1, k = q / n1;
    const long long t = ((k + p.go[2]) * p.np[1] + (j + p.go[1])) * p.np[0] + (i + p.go[0]);
    prim_cell<DIM, NS>(p, t, U, Tin, Tout, Q, flags, do_cfl, s_cfl, s_nu);
  }
  if (do_cfl) block_max2(s_cfl, s_nu, red);
}

// Ghost cells among the padded cells [t0, t1): a copy of the per-cell fields
// of the interior cell that the boundary conditions map them to, with the
// normal velocity and momentum negated across a symmetric boundary (and with
// them the normal u/2, while |u - c|/2 and |u + c|/2 trade places) -- bitwise
// what prim_cell computes for the ghost itself from the mapped conserved
// state (its Newton solve starts from the same warm start and the negation
// commutes with every rounding), at the cost of a copy. The nodal gradients
// are not copied: k_grad computes them over the whole padded block.
template <int DIM, int NS>
__global__ void __launch_bounds__(256)
k_ghost(const __grid_constant__ Params p, double* __restrict__ Q, long long t0, long long t1) {
  using L = Lay<DIM, NS>;
  const long long t = t0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= t1) return;
  const int ip = (int)(t % p.np[0]);
  const int jp = (int)((t / p.np[0]) % p.np[1]);
  const int kp = (int)(t / ((long long)p.np[0] * p.np[1]));
  const int i = ip - p.go[0], j = jp - p.go[1], k = kp - p.go[2];
  bool f[3] = {false, false, false};
  const int si = map_axis(i, p.n[0], p.bc[0][0], p.bc[0][1], &f[0]);
  const int sj = DIM > 1 ? map_axis(j, p.n[1], p.bc[1][0], p.bc[1][1], &f[1]) : 0;
  const int sk = DIM > 2 ? map_axis(k, p.n[2], p.bc[2][0], p.bc[2][1], &f[2]) : 0;
  if (si == i && sj == j && sk == k) return;  // interior
  const long long PC = p.pcells;
  const long long src = ((long long)(sk + p.go[2]) * p.np[1] + (sj + p.go[1])) * p.np[0] +
                        (si + p.go[0]);
#pragma unroll
  for (int v = 0; v < L::GU; ++v) {
    int sv = v;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (f[a] && v == L::AM + a) sv = L::AP + a;
      if (f[a] && v == L::AP + a) sv = L::AM + a;
    }
    double x = Q[sv * PC + src];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
      if (f[a] && (v == L::U + 1 + a || v == L::UN + a || v == L::HU + a)) x = -x;
    Q[v * PC + t] = x;
  }
  if (p.diffusion == 1) {
#pragma unroll
    for (int s = 0; s < NS; ++s) Q[(L::DS + s) * PC + t] = Q[(L::DS + s) * PC + src];
  }
}

// dt from the reduced maxima: CFL / max sum_d (|u_d| + c)/dx_d, and the
// viscous limit CFL dx_min^2 / (2 dim max nu).
__device__ __forceinline__ double dt_from_red(const Params& p, const unsigned long long* red) {
  const double smax = __longlong_as_double((long long)red[0]);
  const double numax = __longlong_as_double((long long)red[1]);
  double dt = p.cfl / smax;
  if (p.viscous && numax > 0.0) dt = fmin(dt, p.cfl * p.hmin2_over_2dim / numax);
  return dt;
}


// ================================================================ k_grad ===
// Nodal (1,-8,0,8,-1)/(12 dx) velocity derivatives along every active axis b,
// wherever the +-2 neighbours along b lie inside the padded box.
template <int DIM, int NS>
__device__ __forceinline__ void grad_cell(const Params& p, long long t, double* __restrict__ Q) {
  using L = Lay<DIM, NS>;
  const long long PC = p.pcells;
  int idx[3];
  {
    const unsigned tu = (unsigned)t, m0 = (unsigned)p.np[0], m1 = (unsigned)p.np[1];
    const unsigned q0 = tu / m0;
    idx[0] = (int)(tu - q0 * m0);
    idx[1] = (int)(q0 % m1);
    idx[2] = (int)(q0 / m1);
  }
  const long long stride[3] = {1, p.np[0], (long long)p.np[0] * p.np[1]};
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    if (idx[b] < 2 || idx[b] >= p.np[b] - 2) continue;
    const long long sb = stride[b];
    const double w = p.inv_dx[b] * (1.0 / 12.0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const double* ua = Q + (L::UN + a) * PC + t;
      const double g = ((ld(ua - 2 * sb) - ld(ua + 2 * sb)) + 8.0 * (ld(ua + sb) - ld(ua - sb))) * w;
      Q[(L::GU + a * DIM + b) * PC + t] = g;
    }
  }
}

template <int DIM, int NS>
__global__ void __launch_bounds__(256)
k_grad(const __grid_constant__ Params p, double* __restrict__ Q) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < p.pcells) grad_cell<DIM, NS>(p, t, Q);
}

// ================================================================= WENO5 ===
// WENO5-JS at i+1/2 from f0..f4 = f_{i-2..i+2}, returned as F = f2 + num/(6 den).
// Written on first differences a..d: the smoothness indicators are scaled by
// 12 (12 b_k = 13 t_k^2 + 3 u_k^2, with 12 eps) -- a common factor that leaves
// the weights unchanged -- and the nonlinear weights d_k/(eps + b_k)^2 are
// scaled by prod_j (eps + b_j)^2, so no division is needed until the end.
// The linear weights d = (0.1, 0.6, 0.3) are folded into the indicators:
// with s_k scaled by c_k proportional to (d_i d_j / d_k)^(1/4)
// ({i, j, k} = {0, 1, 2}), (s_i s_j)^2 already carries the factor d_k. The
// common factor is chosen so that c_0 = 1/16: then c_1 = 1/(16 sqrt 6),
// c_2 = 1/(16 sqrt 3), and the leading square of s_0 has coefficient 1.
// The candidates enter as q_k - f2.
// Each 12 b_k is a positive definite quadratic form in two differences,
// evaluated as its LDL^T sum of squares (exact in these rationals):
//   12 b_0 = 16 a^2 - 44 ab + 40 b^2 = 16 (a - 11/8 b)^2 + 39/4 b^2
//   12 b_1 = 16 b^2 - 20 bc + 16 c^2 = 16 (b - 5/8 c)^2 + 39/4 c^2
//   12 b_2 = 40 c^2 - 44 cd + 16 d^2 = 16 (d - 11/8 c)^2 + 39/4 c^2
// (b_1 and b_2 share c^2).
constexpr double kWc0 = 0.0625;               // 1/16
constexpr double kWc1 = 0.02551551815399144;  // 1/(16 sqrt 6)
constexpr double kWc2 = 0.03608439182435161;  // 1/(16 sqrt 3)

// The face kernel's fixed coefficients, in the order Params::kface holds
// them: the WENO5 indicators' and candidates' (0-10, weno5_nd), the face
// stencil's 9 and 15 (11, 12, face_one), the Newton-Raphson 1 (13), [14: the
// division scale], 1/2 (15), the viscous flux's 1/16, 1/12, 16, 4/3, -2/3
// and 1/256 (16-21, face_one), and the WENO5 adjoint's 6, 32 c_1, 32 c_2,
// 19.5 c_0, 19.5 c_1, 19.5 c_2 (22-27, w5_fwd / w5_rev).
constexpr int kFaceCoefN = 28;
constexpr double kFaceCoef[kFaceCoefN] = {-1.375, -0.625, 9.75 * kWc0, 16.0 * kWc1, 9.75 * kWc1,
                                          16.0 * kWc2, 9.75 * kWc2, -2.0, 2.25, 2.0, 4.0,
                                          9.0, 15.0, 1.0, 0.0, 0.5,
                                          1.0 / 16.0, 1.0 / 12.0, 16.0, 4.0 / 3.0, -2.0 / 3.0,
                                          1.0 / 256.0,
                                          6.0, 32.0 * kWc1, 32.0 * kWc2, 19.5 * kWc0, 19.5 * kWc1,
                                          19.5 * kWc2};

// K = kface in registers, E = {12 eps c_k} in device memory (per call)
__device__ __forceinline__ void weno5_nd(double f0, double f1, double f2, double f3, double f4,
                                         const double* K, const double* E, double& num,
                                         double& den) {
  const double a = f1 - f0, b = f2 - f1, c = f3 - f2, d = f4 - f3;
  const double A0 = fma(K[0], b, a), B1 = fma(K[1], c, b), D2 = fma(K[0], c, d);
  const double cc = c * c;
  const double s0 = fma(A0, A0, fma(K[2] * b, b, __ldcg(E + 0)));  // 16 c_0 = 1
  const double s1 = fma(K[3] * B1, B1, fma(K[4], cc, __ldcg(E + 1)));
  const double s2 = fma(K[5] * D2, D2, fma(K[6], cc, __ldcg(E + 2)));
  // 6 (q_k - f2): 5b - 2a = 9/4 b - 2 A0, 2c + b, 4c - d; the factor 6 goes
  // to the denominator of the field pair (rec_scale)
  const double q0 = fma(K[7], A0, K[8] * b);
  const double q1 = fma(K[9], c, b);
  const double q2 = fma(K[10], c, -d);
  // weights w_0 = (s_1 s_2)^2, w_1 = (s_0 s_2)^2, w_2 = (s_0 s_1)^2 with
  // a_k = s_k^2 grouped as num = a_2 (a_1 q_0 + a_0 q_1) + a_0 a_1 q_2 and
  // den = a_2 (a_0 + a_1) + a_0 a_1
  const double a0 = s0 * s0, a1 = s1 * s1, a2 = s2 * s2;
  const double a01 = a0 * a1;
  num = fma(a2, fma(a1, q0, a0 * q1), a01 * q2);
  den = fma(a2, a0 + a1, a01);
}


// WENO-CU6 (central-upwind, ref. 34): candidates q_0..q_2 of WENO5 and the
// downwind q_3 on {i+1, i+2, i+3}, linear weights (1, 9, 9, 1)/20, beta_3 the
// Jiang-Shu indicator beta_6 of the degree-5 polynomial on all six cells,
// tau = beta_6 - (beta_0 + beta_2 + 4 beta_1)/6 and
// alpha_k = d_k (C + tau/(beta_k + eps)), C = 20.
// Everything is scaled by 12 as in WENO5 and multiplied through by
// prod_j s_j (s_j = 12 (beta_j + eps)): alpha_k ~ d_k (C s_k + 12 tau) prod_{j!=k} s_j,
// so one division per field pair remains. beta_6 is evaluated on the first
// differences x = (f1-f0, .., f5-f4) as sum_k D_k y_k^2, y = L^T x, the LDL^T
// factorisation of its quadratic form (exact rationals, rounded to double);
// on differences it keeps its digits on smooth data with a large offset.
constexpr double kB6D[5] = {12.0 * 2.2468501984126985, 12.0 * 3.6320275079835525,
                            12.0 * 4.2138861378223531, 12.0 * 1.0316113515772065,
                            12.0 * 0.038978122273068759};
constexpr double kB6L10 = -3.3800293620919937, kB6L20 = 4.1377553085411307,
                 kB6L30 = -2.2318538224071762, kB6L40 = 0.45187450097321719;
constexpr double kB6L21 = -1.8788632502196132, kB6L31 = 1.2398246217680282,
                 kB6L41 = -0.28359452031236648;
constexpr double kB6L32 = -0.86413844801584661, kB6L42 = 0.22441845180562248;
constexpr double kB6L43 = -0.38419782506660333;

// e12 = 12 eps
__device__ __forceinline__ void cu6_nd(double f0, double f1, double f2, double f3, double f4,
                                       double f5, double e12, double& num, double& den) {
  const double a = f1 - f0, b = f2 - f1, c = f3 - f2, d = f4 - f3, e = f5 - f4;
  // 12 beta_0..2 as the sums of squares of weno5_nd
  const double A0 = fma(-1.375, b, a), B1 = fma(-0.625, c, b), D2 = fma(-1.375, c, d);
  const double c975 = 9.75 * c * c;
  const double b0 = fma(16.0 * A0, A0, (9.75 * b) * b);
  const double b1 = fma(16.0 * B1, B1, c975);
  const double b2 = fma(16.0 * D2, D2, c975);
  const double y4 = e;
  const double y3 = fma(kB6L43, e, d);
  const double y2 = fma(kB6L42, e, fma(kB6L32, d, c));
  const double y1 = fma(kB6L41, e, fma(kB6L31, d, fma(kB6L21, c, b)));
  const double y0 = fma(kB6L40, e, fma(kB6L30, d, fma(kB6L20, c, fma(kB6L10, b, a))));
  const double b6 = fma(kB6D[0] * y0, y0, fma(kB6D[1] * y1, y1, fma(kB6D[2] * y2, y2,
                    fma(kB6D[3] * y3, y3, kB6D[4] * y4 * y4))));
  const double tau = b6 - (b0 + b2 + 4.0 * b1) * (1.0 / 6.0);   // 12 tau
  const double s0 = b0 + e12, s1 = b1 + e12, s2 = b2 + e12, s3 = b6 + e12;
  const double p01 = s0 * s1, p23 = s2 * s3;
  const double t05 = 0.05 * tau, t45 = 0.45 * tau;   // d_k tau
  const double w0 = fma(0.05 * 20.0, s0, t05) * (s1 * p23);
  const double w1 = fma(0.45 * 20.0, s1, t45) * (s0 * p23);
  const double w2 = fma(0.45 * 20.0, s2, t45) * (p01 * s3);
  const double w3 = fma(0.05 * 20.0, s3, t05) * (p01 * s2);
  // 6 (q_k - f2), as in weno5_nd; q_3: 6c - 5d + 2e
  const double q0 = fma(-2.0, A0, 2.25 * b);
  const double q1 = fma(2.0, c, b);
  const double q2 = fma(4.0, c, -d);
  const double q3 = fma(6.0, c, fma(-5.0, d, 2.0 * e));
  num = fma(w0, q0, fma(w1, q1, fma(w2, q2, w3 * q3)));
  den = (w0 + w1) + (w2 + w3);
}


// WENO7-JS (ref. 36) at i+1/2 from f0..f6 = f_{i-3..i+3}: cubic candidates on
// {i-3+k .. i+k}, linear weights d = (1, 12, 18, 4)/35, Jiang-Shu indicators
// of the cubics. As in WENO5, the indicators are scaled (by 240) and written
// on first differences x_j = f_{j+1} - f_j, as the LDL^T sums of squares of
// their quadratic forms: 240 beta_0 = Q0(x0, x1, x2), 240 beta_1 = Q1(x1, x2, x3),
// and by mirror symmetry 240 beta_2 = Q1(x4, x3, x2), 240 beta_3 = Q0(x5, x4, x3).
// The weights d_k/(eps + beta_k)^2 are multiplied through by prod_j s_j^2;
// scaling s_k by c_k = (35/d_k)^(1/2) makes prod_{j!=k} s_j^2 carry d_k.
constexpr double kW7c0 = 5.9160797830996161, kW7c1 = 1.707825127659933,
                 kW7c2 = 1.3944333775567925, kW7c3 = 2.9580398915498081;
// z2 = 191.02539981185325 y2^2, the last square of both forms (shared by the
// two indicators that end on the same difference)
constexpr double kW7D3 = 191.02539981185325;
__device__ __forceinline__ double w7_q0(double y0, double y1, double y2, double z2) {
  const double A = fma(1.6946983546617915, y2, fma(-2.5484460694698354, y1, y0));
  const double B = fma(-1.4896519285042333, y2, y1);
  return fma(547.0 * A, A, fma(155.46617915904935 * B, B, z2));
}
__device__ __forceinline__ double w7_q1(double y0, double y1, double y2, double z2) {
  const double A = fma(0.92509363295880154, y2, fma(-2.0749063670411987, y1, y0));
  const double B = fma(-0.6326434619002822, y2, y1);
  return fma(267.0 * A, A, fma(318.50187265917606 * B, B, z2));
}

// ec[k] = 240 eps c_k
__device__ __forceinline__ void weno7_nd(double f0, double f1, double f2, double f3, double f4,
                                         double f5, double f6, const double* ec, double& num,
                                         double& den) {
  const double x0 = f1 - f0, x1 = f2 - f1, x2 = f3 - f2, x3 = f4 - f3, x4 = f5 - f4,
               x5 = f6 - f5;
  const double z2 = kW7D3 * x2 * x2, z3 = kW7D3 * x3 * x3;
  const double s0 = fma(kW7c0, w7_q0(x0, x1, x2, z2), ec[0]);
  const double s1 = fma(kW7c1, w7_q1(x1, x2, x3, z3), ec[1]);
  const double s2 = fma(kW7c2, w7_q1(x4, x3, x2, z2), ec[2]);
  const double s3 = fma(kW7c3, w7_q0(x5, x4, x3, z3), ec[3]);
  const double p01 = s0 * s1, p23 = s2 * s3;
  const double r0 = s1 * p23, r1 = s0 * p23, r2 = p01 * s3, r3 = p01 * s2;
  const double w0 = r0 * r0, w1 = r1 * r1, w2 = r2 * r2, w3 = r3 * r3;
  // candidates minus f3
  const double q0 = fma(0.25, x0, fma(-5.0 / 6.0, x1, (13.0 / 12.0) * x2));
  const double q1 = fma(-1.0 / 12.0, x1, fma(1.0 / 3.0, x2, 0.25 * x3));
  const double q2 = fma(1.0 / 12.0, x2, fma(0.5, x3, (-1.0 / 12.0) * x4));
  const double q3 = fma(0.75, x3, fma(-1.0 / 3.0, x4, (1.0 / 12.0) * x5));
  num = fma(w0, q0, fma(w1, q1, fma(w2, q2, w3 * q3)));
  den = (w0 + w1) + (w2 + w3);
}

// F^+ + F^- of one characteristic field (Eq. 15) with the reconstruction REC
// (5: WENO5-JS, 6: WENO-CU6, 7: WENO7-JS): the upwind reconstruction of w^+
// and the mirrored one of w^- about the face, as b + n/d with the division
// left to the caller (two fields share one). Stencils: w^+ from i-2..i+2
// (i-3..i+3 for WENO7, i-2..i+3 for CU6), w^- mirrored from i+3 (i+4).
// e4 = {12 eps c_0, 12 eps c_1, 12 eps c_2, 12 eps} for 5 and 6, {240 eps c_k}
// for 7; WENO5 takes its coefficients K (registers) and its eps E (device
// memory) instead.
struct RecND {
  double b, n, d;
};
template <int REC>
__device__ __forceinline__ RecND rec_nd(const double* wp, const double* wm, const double* e4,
                                        const double* K, const double* E) {
  double np, dp, nm, dm, b;
  if constexpr (REC == 7) {
    weno7_nd(wp[0], wp[1], wp[2], wp[3], wp[4], wp[5], wp[6], e4, np, dp);
    weno7_nd(wm[7], wm[6], wm[5], wm[4], wm[3], wm[2], wm[1], e4, nm, dm);
    b = wp[3] + wm[4];
  } else if constexpr (REC == 6) {
    cu6_nd(wp[0], wp[1], wp[2], wp[3], wp[4], wp[5], e4[3], np, dp);
    cu6_nd(wm[5], wm[4], wm[3], wm[2], wm[1], wm[0], e4[3], nm, dm);
    b = wp[2] + wm[3];
  } else {
    weno5_nd(wp[0], wp[1], wp[2], wp[3], wp[4], K, E, np, dp);
    weno5_nd(wm[5], wm[4], wm[3], wm[2], wm[1], K, E, nm, dm);
    b = wp[2] + wm[3];
  }
  return RecND{b, fma(np, dm, nm * dp), dp * dm};
}
// the WENO5 and CU6 numerators carry a factor 6 (weno5_nd, cu6_nd), taken
// out at the division
template <int REC>
__host__ __device__ constexpr double rec_scale() { return REC == 7 ? 1.0 : 6.0; }
// K[13] = 1, K[14] = rec_scale<REC>() (registers)
template <int REC>
__device__ __forceinline__ double rec_div1(const RecND& x, const double* K) {
  return fma(x.n, rcp_nr1(K[14] * x.d, K[13]), x.b);
}
// two fields with one division: 1/d_x = d_y / (d_x d_y). The weights are
// scaled by the indicators' products (section above), so d_x d_y stays far
// inside the double range for any finite stencil data the solver meets.
template <int REC>
__device__ __forceinline__ void rec_div2(const RecND& x, const RecND& y, double& fx, double& fy,
                                         const double* K) {
  const double r = rcp_nr1((K[14] * x.d) * y.d, K[13]);
  fx = fma(x.n, r * y.d, x.b);
  fy = fma(y.n, r * x.d, y.b);
}

// ================================================================= k_face ===
// One thread per face of direction D (faces i = 0..n_D, left cell i-1).
#ifndef XF_FACE_THREADS
#define XF_FACE_THREADS 128
#endif
#ifndef XF_FACE_MIN_BLOCKS
#define XF_FACE_MIN_BLOCKS (256 / XF_FACE_THREADS)
#endif
// Convective face flux of Eq. 15 (Roe-averaged face state, PER projection,
// LLF splitting of Eq. 14, reconstruction REC, back-projection) into Gout,
// for the face between the cells q0 and q0 + sd (stride of direction D).
template <int DIM, int NS, int D, int REC>
__device__ __forceinline__ void conv_flux(const Params& p, const double* __restrict__ q0,
                                          long long PC, long long sd, double* Gout,
                                          uint32_t& st) {
  using L = Lay<DIM, NS>;
  constexpr int SO = REC == 7 ? 3 : 2;  // stencil cells left of the left cell
  constexpr int SW = 2 * SO + 2;        // stencil width
  constexpr int IE = DIM + 1;
#define QF(field, m) ld(q0 + (long long)(field) * PC + (long long)(m) * sd)
  // ---- Roe-averaged face state (sqrt(rho) weights)
  const double sL = QF(L::SR, 0), sR = QF(L::SR, 1);
  const double one = __ldcg(p.dev->kface + 13), half = __ldcg(p.dev->kface + 15);
  const double iw = rcp_nr1(sL + sR, one);
  const double tL = sL * iw, tR = sR * iw;
  double ub[DIM], q2 = 0.0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    ub[a] = fma(tL, QF(L::UN + a, 0), tR * QF(L::UN + a, 1));
    q2 = fma(ub[a], ub[a], q2);
  }
  const double Hb = fma(tL, QF(L::H, 0), tR * QF(L::H, 1));
  const double Tb = fma(tL, QF(L::T, 0), tR * QF(L::T, 1));
  double Yb[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) Yb[s] = fma(tL, QF(L::Y + s, 0), tR * QF(L::Y + s, 1));
  const TauPt tp = tau_pt(p, fma(Tb, rd(p.dev->inv_span), rd(p.dev->tau0)));
  // h_N and h_s - h_N (s = 1..N-1): the species' eigenvectors need phi_s - phi_N only
  const double hN = h_s_dev(p, NS - 1, tp);
  double hd[NS > 1 ? NS - 1 : 1];
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) hd[s] = hd_s_dev(p, s, tp);
  // R(Y) and c_p(Y, T) are linear in Y: their face values come from the two
  // cells' mixture gas constants and c_p coefficients with the same weights
  const double Rb = fma(tL, QF(L::RM, 0), tR * QF(L::RM, 1));
  double Ab[5];
#pragma unroll
  for (int jj = 0; jj < 5; ++jj) Ab[jj] = fma(tL, QF(L::AC + jj, 0), tR * QF(L::AC + jj, 1));
  const double cpb = fma(fma(fma(fma(Ab[4], tp.tc, Ab[3]), tp.tc, Ab[2]), tp.tc, Ab[1]), tp.tc, Ab[0]);
  const double cvb = cpb - Rb;
  // one division for Gamma = R/c_v and its inverse
  const double rRc = rcp_nr1(Rb * cvb, one);
  const double Gam = Rb * Rb * rRc;
  const double hq2 = half * q2;
  // phi_s = R_s T - Gamma (e_s - |u|^2/2) with e_s = h_s - R_s T:
  // R_s (1 + Gamma) T - Gamma h_s + Gamma |u|^2/2; formed as phi_N and
  // phi_s - phi_N = (R_s - R_N)(1 + Gamma) T - Gamma (h_s - h_N), and with
  // sum_s Y_s = 1, sum_s Y_s phi_s = phi_N + sum_{s<N} Y_s (phi_s - phi_N)
  const double T1G = fma(Gam, Tb, Tb), Gq2 = Gam * hq2;
  const double phiN = fma(__ldcg(p.dev->r + NS - 1), T1G, fma(-Gam, hN, Gq2));
  double dphi[NS > 1 ? NS - 1 : 1], c2 = phiN;
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) {
    dphi[s] = fma(__ldcg(p.dev->rdN + s), T1G, -Gam * hd[s]);
    c2 = fma(Yb[s], dphi[s], c2);
  }
  c2 = fma(Gam, Hb - q2, c2);
  if (!(c2 > 0.0)) {
    st |= 4u;
    const double cl = QF(L::C, 0), cr = QF(L::C, 1);
    c2 = 0.5 * (cl * cl + cr * cr);
  }
  const double rsc = rsqrt(c2);
  const double c = c2 * rsc;
  const double ic2 = rsc * rsc;
  const double hic2 = half * ic2;
  const double iGam = cvb * cvb * rRc;
  const double un = ub[D];
  // ---- stencil m = i-SO..i+SO+1 (SW cells: i-2..i+3 for WENO5 and CU6,
  //      i-3..i+4 for WENO7; offsets from the left cell). Per cell:
  //      rho, p, u_n/2, g.U/(2c^2) and the LLF maxima of |u-c|/2, |u+c|/2,
  //      |u|/2 (the halves stored by primitive recovery: exactly half the
  //      maxima of |u-c|, |u+c|, |u|). The 1/2 of Eq. 14 and the 1/(2c^2)
  //      of the acoustic rows are folded into per-face coefficients.
  const double gE = Gam * hic2;
  double gm[DIM], gs[NS > 1 ? NS - 1 : 1];
#pragma unroll
  for (int a = 0; a < DIM; ++a) gm[a] = -ub[a] * gE;
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) gs[s] = dphi[s] * hic2;
  const double gr = phiN * hic2;
  double rho_m[SW], p_m[SW], hun[SW], gUh[SW];
  double ham = 0.0, hap = 0.0, ha0 = 0.0;
#pragma unroll
  for (int m = 0; m < SW; ++m) {
    const int o = m - SO;
    rho_m[m] = QF(L::U, o);
    hun[m] = QF(L::HU + D, o);
    p_m[m] = QF(L::P, o);
    ham = pmax(ham, QF(L::AM + D, o));
    hap = pmax(hap, QF(L::AP + D, o));
    ha0 = pmax(ha0, fabs(hun[m]));
    double g = gr * rho_m[m];
#pragma unroll
    for (int a = 0; a < DIM; ++a) g = fma(gm[a], QF(L::U + 1 + a, o), g);
    g = fma(gE, QF(L::U + IE, o), g);
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) g = fma(gs[s], QF(L::U + IE + 1 + s, o), g);
    gUh[m] = g;
  }
  const double e12c[4] = {p.wenoe[0], p.wenoe[1], p.wenoe[2], p.wenoe[3]};
  const double e12q[4] = {p.wenoe4[0], p.wenoe4[1], p.wenoe4[2], p.wenoe4[3]};
  double K[15];
#pragma unroll
  for (int j = 0; j < 15; ++j) K[j] = __ldcg(p.dev->kface + j);
  const double* Ec = p.dev->wenoe;
  const double* Eq = p.dev->wenoe4;
  const double chc = c * hic2;
  // ---- PER: one characteristic field at a time. With w = (1/2)(l.F_m +- a l.U_m)
  //      and l.F_m = u_m (l.U_m) + p_m (l[m_n] + u_m l[E]):
  //      w^+- = (u_m/2 +- a/2) l.U_m + p_m (l[m_n]/2 + (u_m/2) l[E]).
  // the passive fields (eigenvalue u, no pressure term): tangential momenta,
  // l = (-u_t, e_{m_t}), r = e_{m_t} + u_t e_E; species, l = (-Y_s, e_{rhoY_s}),
  // r = e_{rhoY_s} - (phi_s - phi_N)/Gamma e_E. Passive field k < DIM-1 is the
  // tangential axis k (skipping D), the rest the species k - (DIM-1).
  constexpr int NPASS = DIM - 1 + NS - 1;
  double hp0[SW], hm0[SW];
  auto passive_nd = [&](int k) -> RecND {
    double wp[SW], wm[SW];
    if (k < DIM - 1) {
      const int a = k < D ? k : k + 1;
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        const double LU = fma(-ub[a], rho_m[m], QF(L::U + 1 + a, m - SO));
        wp[m] = hp0[m] * LU;
        wm[m] = hm0[m] * LU;
      }
    } else {
      const int s = k - (DIM - 1);
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        const double LU = fma(-Yb[s], rho_m[m], QF(L::U + IE + 1 + s, m - SO));
        wp[m] = hp0[m] * LU;
        wm[m] = hm0[m] * LU;
      }
    }
    return rec_nd<REC>(wp, wm, e12c, K, Ec);
  };
  double Fk_m, Fk_p, Fk_e, Fk_first = 0.0;
  {
    double wp[SW], wm[SW];
    RecND ndm, ndp, nde;
    // normal momentum relative to the face velocity, shared by u -+ c
    double nUv[SW];
#pragma unroll
    for (int m = 0; m < SW; ++m) nUv[m] = fma(-un, rho_m[m], QF(L::U + 1 + D, m - SO));
    // the pressure terms p_m (l[m_n]/2 + (u_m/2) l[E]) of the three dense rows
    // from one product per cell: with lE = Gam/(2c^2) and hl0 = -Gam u_n/(4c^2),
    // the u -+ c rows take p_m (u_m/2 lE + hl0 -+ c/(4c^2)) and the entropy row
    // exactly -2 p_m (u_m/2 lE + hl0)
    const double lE = gE, hl0 = (-half * un) * gE, dl = half * chc;
    double pV[SW];
#pragma unroll
    for (int m = 0; m < SW; ++m) pV[m] = p_m[m] * fma(hun[m], lE, hl0);
    // u - c: l.U = (g.U - c (m_n - u_n rho)) / (2c^2)
    {
      const double ha = ham;
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        const double LU = fma(-chc, nUv[m], gUh[m]);
        const double X = fma(hun[m], LU, fma(-dl, p_m[m], pV[m]));
        wp[m] = fma(ha, LU, X);
        wm[m] = fma(-ha, LU, X);
      }
      ndm = rec_nd<REC>(wp, wm, e12c, K, Ec);
    }
    // u + c
    {
      const double ha = hap;
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        const double LU = fma(chc, nUv[m], gUh[m]);
        const double X = fma(hun[m], LU, fma(dl, p_m[m], pV[m]));
        wp[m] = fma(ha, LU, X);
        wm[m] = fma(-ha, LU, X);
      }
      ndp = rec_nd<REC>(wp, wm, e12c, K, Ec);
    }
    rec_div2<REC>(ndm, ndp, Fk_m, Fk_p, K);
    // (u_m +- |u|max)/2, shared by the entropy row and the passive fields
#pragma unroll
    for (int m = 0; m < SW; ++m) { hp0[m] = hun[m] + ha0; hm0[m] = hun[m] - ha0; }
    // entropy: l = e_rho - g / c^2, w = (u_m/2 +- a/2)(rho - 2 g.U/(2c^2)) - 2 pV,
    // reconstructed as -w/2 = (u_m/2 +- a/2)(g.U/(2c^2) - rho/2) + pV with
    // eps/4 (bitwise -1/2 of the reconstruction of w: a power-of-two factor
    // commutes with every rounding); Fk_eh is -Fk_e/2
    {
#pragma unroll
      for (int m = 0; m < SW; ++m) {
        const double LUh = fma(-half, rho_m[m], gUh[m]);
        wp[m] = fma(hp0[m], LUh, pV[m]);
        wm[m] = fma(hm0[m], LUh, pV[m]);
      }
      nde = rec_nd<REC>(wp, wm, e12q, K, Eq);
    }
    // the entropy field shares its division with the first passive field
    if constexpr (NPASS > 0) rec_div2<REC>(nde, passive_nd(0), Fk_e, Fk_first, K);
    else Fk_e = rec_div1<REC>(nde, K);
  }
  // back-projection of the three dense right columns (Eq. 15)
  {
    const double S = fma(K[7], Fk_e, Fk_m + Fk_p);  // K[7] = -2
    const double Dl = Fk_p - Fk_m;
    Gout[0] = S;
#pragma unroll
    for (int a = 0; a < DIM; ++a) Gout[1 + a] = ub[a] * S;
    Gout[1 + D] = fma(c, Dl, Gout[1 + D]);
    Gout[IE] = fma(Hb, S, fma(un * c, Dl, (c2 + c2) * iGam * Fk_e));
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) Gout[IE + 1 + s] = Yb[s] * S;
  }
  // the passive fields' right columns, in order, two fields per division
  auto passive_add = [&](int k, double Fk) {
    if (k < DIM - 1) {
      const int a = k < D ? k : k + 1;
      Gout[1 + a] += Fk;
      Gout[IE] = fma(ub[a], Fk, Gout[IE]);
    } else {
      const int s = k - (DIM - 1);
      Gout[IE + 1 + s] += Fk;
      Gout[IE] = fma(-dphi[s] * iGam, Fk, Gout[IE]);
    }
  };
  if constexpr (NPASS > 0) passive_add(0, Fk_first);
#pragma unroll
  for (int k = 1; k < NPASS; k += 2) {
    const RecND x = passive_nd(k);
    if (k + 1 < NPASS) {
      double fx, fy;
      rec_div2<REC>(x, passive_nd(k + 1), fx, fy, K);
      passive_add(k, fx);
      passive_add(k + 1, fy);
    } else {
      passive_add(k, rec_div1<REC>(x, K));
    }
  }
#undef QF
}

// Positivity-preserving blend of one face's convective flux Gout (in place),
// for the face between the cells q0 and q0 + sd; dt is the stage time step.
template <int DIM, int NS, int D>
__device__ __forceinline__ void pos_blend(const Params& p, const double* __restrict__ q0,
                                          long long PC, long long sd, double dt, double* Gout) {
  using L = Lay<DIM, NS>;
  constexpr int NV = L::NV;
  constexpr int IE = DIM + 1;
#define QF(field, m) ld(q0 + (long long)(field) * PC + (long long)(m) * sd)
  // Positivity-preserving blend (Eq. 17-20): F* = (1 - theta) F_LF + theta F_hat
  // with the local LF flux of Eq. 19 (alpha = max(|u_d| + c) of the two cells);
  // theta keeps every partial density of U_i - 2 lam F* and U_{i+1} + 2 lam F*
  // (Eq. 18, lam = dim dt / dx_d) at or above min(pos_eps, its LF value).
  const double lam2 = 2.0 * DIM * dt * p.inv_dx[D];
  double Fa[NV], Fb[NV], Ua[NV], Ub[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { Ua[v] = QF(L::U + v, 0); Ub[v] = QF(L::U + v, 1); }
  const double una = QF(L::UN + D, 0), unb = QF(L::UN + D, 1);
  const double pa = QF(L::P, 0), pb = QF(L::P, 1);
#pragma unroll
  for (int v = 0; v < NV; ++v) { Fa[v] = una * Ua[v]; Fb[v] = unb * Ub[v]; }
  Fa[1 + D] += pa; Fb[1 + D] += pb;
  Fa[IE] += pa * una; Fb[IE] += pb * unb;
  const double al = fmax(fabs(una) + QF(L::C, 0), fabs(unb) + QF(L::C, 1));
  double Flf[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Flf[v] = 0.5 * (Fa[v] + Fb[v] + al * (Ua[v] - Ub[v]));
  double theta = 1.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double qa, qb, fh, fl;
    if (s < NS - 1) {
      qa = Ua[IE + 1 + s]; qb = Ub[IE + 1 + s]; fh = Gout[IE + 1 + s]; fl = Flf[IE + 1 + s];
    } else {
      qa = Ua[0]; qb = Ub[0]; fh = Gout[0]; fl = Flf[0];
#pragma unroll
      for (int k = 0; k < NS - 1; ++k) {
        qa -= Ua[IE + 1 + k]; qb -= Ub[IE + 1 + k]; fh -= Gout[IE + 1 + k]; fl -= Flf[IE + 1 + k];
      }
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const double sg = side == 0 ? -lam2 : lam2;
      const double q = side == 0 ? qa : qb;
      const double hi = fma(sg, fh, q), lo = fma(sg, fl, q);
      const double eps = fmin(lo, p.pos_eps);
      if (hi < eps) theta = fmin(theta, fmax((lo - eps) / (lo - hi), 0.0));
    }
  }
  if (theta < 1.0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Gout[v] = fma(theta, Gout[v] - Flf[v], Flf[v]);
  }
#undef QF
}

// Per-face body: face (fi, fj, fk) of direction D, i.e. between cells
// idx - e_D and idx (fi in 0..n_0 when D = 0, and so on).
// With Fh given, the face's unblended convective flux (Eq. 15, before the
// blend and the viscous terms) also goes to Fh ([n_v][faces], Gf's layout).
template <int DIM, int NS, int D, int REC = 5>
__device__ __forceinline__ void face_one(const Params& p, int fi, int fj, int fk,
                                         const double* __restrict__ Q, double* __restrict__ Gf,
                                         uint32_t* __restrict__ flags, double dt,
                                         double* __restrict__ Fh = nullptr) {
  using L = Lay<DIM, NS>;
  constexpr int NV = L::NV;
  constexpr int IE = DIM + 1;
  const int nf0 = p.n[0] + (D == 0), nf1 = p.n[1] + (D == 1), nf2 = p.n[2] + (D == 2);
  const long long nfaces = (long long)nf0 * nf1 * nf2;
  const long long f = ((long long)fk * nf1 + fj) * nf0 + fi;
  int id[3] = {fi, fj, fk};
  id[D] -= 1;  // left cell
  const long long PC = p.pcells;
  const long long sy = p.np[0], sz = (long long)p.np[0] * p.np[1];
  const long long c0 = (id[2] + p.go[2]) * sz + (id[1] + p.go[1]) * sy + (id[0] + p.go[0]);
  const long long sd = D == 0 ? 1 : (D == 1 ? sy : sz);
  const double* q0 = Q + c0;
#define QF(field, m) ld(q0 + (long long)(field) * PC + (long long)(m) * sd)
  double Gout[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Gout[v] = 0.0;
  uint32_t st = 0;

  if (p.convective) conv_flux<DIM, NS, D, REC>(p, q0, PC, sd, Gout, st);
  if (Fh) {
#pragma unroll
    for (int v = 0; v < NV; ++v) Fh[v * nfaces + f] = Gout[v];
  }

  if (p.convective && p.positivity && dt > 0.0) pos_blend<DIM, NS, D>(p, q0, PC, sd, dt, Gout);

  if (p.viscous) {
    // face values (-1, 9, 9, -1)/16, normal derivatives (1, -15, 15, -1)/(12 dx).
    // FI0 / FD0 leave out the factors 1/16 and 1/(12 dx); each product below
    // takes them once (wi, wd, wid = wi wd). The constants come from the
    // parameters' device copy (register operands).
    const double* kf = p.dev->kface;
    const double wi = rd(kf[16]);
    const double wd = rd(p.dev->inv_dx[D]) * rd(kf[17]);
    const double wid = wi * wd;
    const double k9 = rd(kf[11]), k15 = rd(kf[12]);
#define FI0(field) (fma(k9, QF(field, 0) + QF(field, 1), -(QF(field, -1) + QF(field, 2))))
#define FD0(field) (fma(k15, QF(field, 1) - QF(field, 0), -(QF(field, 2) - QF(field, -1))))
    // tau_Da (Eq. 3) = (mu/16) t16_a with t16_a = 16 (du_D/dx_a + du_a/dx_D)
    // for a != D and t16_D = 16 (4/3 du_D/dx_D - 2/3 sum_{a != D} du_a/dx_a);
    // FI0 of the nodal derivatives is 16 times their face value, FD0 of u is
    // the normal derivative over wd, so rq = wd/wi weights the normal ones
    const double mu16 = FI0(L::MU) * rd(kf[21]);  // wi wi
    const double rq = rd(kf[18]) * wd;
    double t16[DIM], tr = 0.0;
    bool first = true;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (a == D) continue;
      t16[a] = fma(rq, FD0(L::UN + a), FI0(L::GU + D * DIM + a));
      tr = first ? FI0(L::GU + a * DIM + a) : tr + FI0(L::GU + a * DIM + a);
      first = false;
    }
    t16[D] = fma(rd(kf[19]) * rq, FD0(L::UN + D), rd(kf[20]) * tr);  // 4/3, -2/3
    // 256 sum_a tau_a u_a / mu16 = sum_a t16_a FI0(u_a); products that feed
    // a sum are written as fused multiply-adds, here and below, so the
    // batched kernel, which compiles this body too, gives the same bits
    double W = t16[0] * FI0(L::UN);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      Gout[1 + a] = fma(-mu16, t16[a], Gout[1 + a]);
      if (a > 0) W = fma(t16[a], FI0(L::UN + a), W);
    }
    // species fluxes of Eq. 6 with the mixture correction, J_s = nJ Jn_s.
    // With dY0 = 12 dx dY/dn, Yf0 = 16 Y_f, Ds0 = 16 D_s and
    // nrf = -rho_f wi wd: D_s = the face values of the cells' D_sm
    // (diffusion = 1): Jn_s = Ds0 dY0_s - Yf0_s wi sum_t Ds0_t dY0_t,
    // nJ = nrf; one D for every species (diffusion = 0): the correction is
    // D Y_s sum_t dY_t/dn = D Y_s d(sum_t Y_t)/dn, identically zero (Y_N is
    // 1 - sum of the others, and the stencil is linear), so Jn_s = dY0_s,
    // nJ = nrf Ds0
    const double nrf = FI0(L::U) * (-wi * wid);
    double Jn[NS], nJ;
    if (p.diffusion == 1) {
      double dY0[NS], Yf0[NS], Ds0[NS];
      double c = 0.0;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        dY0[s] = FD0(L::Y + s); Yf0[s] = FI0(L::Y + s); Ds0[s] = FI0(L::DS + s);
        c = fma(Ds0[s], dY0[s], c);
      }
      const double corr0 = c * wi;
#pragma unroll
      for (int s = 0; s < NS; ++s) Jn[s] = fma(Ds0[s], dY0[s], -Yf0[s] * corr0);
      nJ = nrf;
    } else {
#pragma unroll
      for (int s = 0; s < NS; ++s) Jn[s] = FD0(L::Y + s);
      nJ = nrf * FI0(L::DF);
    }
    // h_s at the face temperature T_f = wi FI0(T); qd = sum_s h_s J_s / nJ.
    // Either model conserves mass, sum_s J_s = 0 (sum_s Y_s = 1 and the
    // stencils are linear), so qd = sum_{s<N} (h_s - h_N) J_s / nJ
    const TauPt tp = tau_pt(p, fma(FI0(L::T), wi * rd(p.dev->inv_span), rd(p.dev->tau0)));
    double qd = 0.0;
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) qd = fma(hd_s_dev(p, s, tp), Jn[s], qd);
    Gout[IE] -= fma(FI0(L::KA) * wid, FD0(L::T), fma(mu16 * wi, W, -nJ * qd));
#pragma unroll
    for (int s = 0; s < NS - 1; ++s) Gout[IE + 1 + s] = fma(nJ, Jn[s], Gout[IE + 1 + s]);
#undef FI0
#undef FD0
  }
#undef QF
#pragma unroll
  for (int v = 0; v < NV; ++v) Gf[v * nfaces + f] = Gout[v];
  raise(flags, st);
}

// Faces [f0, f1) of direction D in their (i fastest) order, f1 <= their count.
template <int DIM, int NS, int D, int REC = 5>
__global__ void __launch_bounds__(XF_FACE_THREADS, XF_FACE_MIN_BLOCKS)
k_face(const __grid_constant__ Params p, const double* __restrict__ Q,
       double* __restrict__ Gf, uint32_t* __restrict__ flags, const double* __restrict__ dtp,
       long long f0, long long f1) {
  const int nf0 = p.n[0] + (D == 0), nf1 = p.n[1] + (D == 1);
  const long long f = f0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= f1) return;
  face_one<DIM, NS, D, REC>(p, (int)(f % nf0), (int)((f / nf0) % nf1), (int)(f / ((long long)nf0 * nf1)),
                       Q, Gf, flags, dtp ? *dtp : 0.0);
}

// Every face of direction D as k_face, also writing the unblended convective
// fluxes to Fh: the tape that the reverse of the positivity blend reads
// (xf_step_rk3_tape_flux) instead of recomputing them.
template <int DIM, int NS, int D, int REC = 5>
__global__ void __launch_bounds__(XF_FACE_THREADS, XF_FACE_MIN_BLOCKS)
k_face_tape(const __grid_constant__ Params p, const double* __restrict__ Q,
            double* __restrict__ Gf, uint32_t* __restrict__ flags, const double* __restrict__ dtp,
            double* __restrict__ Fh) {
  const int nf0 = p.n[0] + (D == 0), nf1 = p.n[1] + (D == 1), nf2 = p.n[2] + (D == 2);
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= (long long)nf0 * nf1 * nf2) return;
  face_one<DIM, NS, D, REC>(p, (int)(f % nf0), (int)((f / nf0) % nf1), (int)(f / ((long long)nf0 * nf1)),
                            Q, Gf, flags, dtp ? *dtp : 0.0, Fh);
}

// =============================================================== k_update ===
// Conservative difference (Eq. 13) and SSP-RK3 (Eq. 16).
//   mode 0: out = L(U)                   (plain RHS)
//   mode 1: out = Un + dt L              (stage 1)
//   mode 2: out = 3/4 Un + 1/4 (Us + dt L)
//   mode 3: out = 1/3 Un + 2/3 (Us + dt L)
template <int DIM, int NS>
__device__ __forceinline__ void update_cell(const Params& p, long long c,
                                            const double* __restrict__ Gx,
                                            const double* __restrict__ Gy,
                                            const double* __restrict__ Gz, const double* Un,
                                            const double* Us, double* out, double dt, int mode) {
  constexpr int NV = DIM + 1 + NS;
  // 32-bit index arithmetic: a handle's padded block holds < 2^31 cells
  const unsigned cu = (unsigned)c, n0 = (unsigned)p.n[0], n1 = (unsigned)p.n[1];
  const unsigned q0 = cu / n0;
  const int i = (int)(cu - q0 * n0);
  const int j = (int)(q0 % n1);
  const int k = (int)(q0 / n1);
  const long long C = p.cells;
  long long fy = 0, fz = 0, NFY = 0, NFZ = 0, sy = 0, sz = 0;
  const long long NFX = (long long)(p.n[0] + 1) * p.n[1] * p.n[2];
  const long long fx = ((long long)k * p.n[1] + j) * (p.n[0] + 1) + i;
  if (DIM > 1) {
    NFY = (long long)p.n[0] * (p.n[1] + 1) * p.n[2];
    fy = ((long long)k * (p.n[1] + 1) + j) * p.n[0] + i;
    sy = p.n[0];
  }
  if (DIM > 2) {
    NFZ = (long long)p.n[0] * p.n[1] * (p.n[2] + 1);
    fz = c;
    sz = (long long)p.n[0] * p.n[1];
  }
  // every input of this cell is read before any output is written: out may be
  // Un or Us (in-place stages), but only at this cell, so the loads of all
  // fields can be in flight together
  double R[NV], un[NV], us[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    R[v] = -(ld(Gx + v * NFX + fx + 1) - ld(Gx + v * NFX + fx)) * p.inv_dx[0];
    if (DIM > 1) R[v] = fma(-(ld(Gy + v * NFY + fy + sy) - ld(Gy + v * NFY + fy)), p.inv_dx[1], R[v]);
    if (DIM > 2) R[v] = fma(-(ld(Gz + v * NFZ + fz + sz) - ld(Gz + v * NFZ + fz)), p.inv_dx[2], R[v]);
    un[v] = mode >= 1 ? Un[v * C + c] : 0.0;
    us[v] = mode >= 2 ? Us[v * C + c] : 0.0;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double o;
    if (mode == 0) {
      o = R[v];
    } else if (mode == 1) {
      o = fma(dt, R[v], un[v]);
    } else if (mode == 2) {
      o = fma(0.75, un[v], 0.25 * fma(dt, R[v], us[v]));
    } else {
      o = fma(1.0 / 3.0, un[v], (2.0 / 3.0) * fma(dt, R[v], us[v]));
    }
    out[v * C + c] = o;
  }
}

// Interior cells [c0, c1), c1 <= cells, with RANGE; every cell without (c0
// and c1 unused: the whole-grid launches keep the plain index, which runs
// faster in this memory-bound kernel).
template <int DIM, int NS, bool RANGE = false>
__global__ void __launch_bounds__(256)
k_update(const __grid_constant__ Params p, const double* __restrict__ Gx,
         const double* __restrict__ Gy, const double* __restrict__ Gz,
         const double* Un, const double* Us, double* out, const double* __restrict__ dtp,
         int mode, long long c0, long long c1) {
  long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (RANGE) {
    c += c0;
    if (c >= c1) return;
  } else {
    if (c >= p.cells) return;
  }
  update_cell<DIM, NS>(p, c, Gx, Gy, Gz, Un, Us, out, mode ? *dtp : 0.0, mode);
}

// ============================================================ k_from_prim ===
// Primitive (rho, u, p, Y) -> conserved U and T with the EOS (Eq. 7).
template <int DIM, int NS>
__global__ void __launch_bounds__(256)
k_from_prim(const __grid_constant__ Params p, const double* __restrict__ P,
            double* __restrict__ U, double* __restrict__ T) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.cells) return;
  const long long C = p.cells;
  const double rho = P[c];
  double Y[NS], ys = 0.0, Rm = 0.0;
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) { Y[s] = P[(DIM + 2 + s) * C + c]; ys += Y[s]; }
  Y[NS - 1] = 1.0 - ys;
#pragma unroll
  for (int s = 0; s < NS; ++s) Rm = fma(Y[s], p.r[s], Rm);
  const double pr = P[(DIM + 1) * C + c];
  const double Tc = pr / (rho * Rm);
  const TauPt tp = tau_of(p, Tc);
  double e = 0.0, ke = 0.0;
#pragma unroll
  for (int s = 0; s < NS; ++s) e = fma(Y[s], h_s(p, s, tp, cp_s(p, s, tp.tc)) - p.r[s] * Tc, e);
  U[c] = rho;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const double u = P[(1 + a) * C + c];
    U[(1 + a) * C + c] = rho * u;
    ke = fma(u, u, ke);
  }
  U[(DIM + 1) * C + c] = rho * fma(0.5, ke, e);
#pragma unroll
  for (int s = 0; s < NS - 1; ++s) U[(DIM + 2 + s) * C + c] = rho * Y[s];
  T[c] = Tc;
}

}  // namespace xf

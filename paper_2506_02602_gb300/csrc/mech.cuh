// mech.cuh -- compile-time structure of the H2-O2-N2 mechanism and the per-context
// coefficient tables the kernels read.
//
// The kernels are specialised to the stoichiometry of a 9-species / 21-reaction
// hydrogen mechanism (Eq. 15): every species index and stoichiometric coefficient is
// a compile-time constant, so the law of mass action (Eq. 16) unrolls into straight
// register code with no per-reaction branching on data.  The coefficients (Arrhenius,
// efficiencies, Troe, NASA-7) are runtime data: chem_setup packs them into MechTables,
// which every launch passes by value as a __grid_constant__ parameter, so the tables
// sit in the constant bank, are read with uniform (broadcast) accesses and need no
// global state -- several contexts with different coefficients can coexist.
#pragma once

#include <cstdint>

namespace chem {

constexpr double R_U = 8.31446261815324;  // J/(mol K)
constexpr double P_REF = 101325.0;        // Pa, standard state of the equilibrium constants

constexpr int NSP = 9;
constexpr int NRX = 21;

// species order of the compiled structure
enum Sp : int { H2 = 0, O2 = 1, H2O = 2, H = 3, O = 4, OH = 5, HO2 = 6, H2O2 = 7, N2 = 8, NONE = -1 };

enum RxType : int { ELEM = 0, THIRD_BODY = 1, FALLOFF = 2 };

// Reaction structure: up to two reactant and two product molecules (a repeated
// species appears twice), reaction type, number of Troe parameters.
struct RxStruct {
  int r0, r1, p0, p1, type, troe_n;
};

constexpr RxStruct kRx[NRX] = {
    {H, O2, O, OH, ELEM, 0},         //  0 H + O2 = O + OH
    {O, H2, H, OH, ELEM, 0},         //  1 O + H2 = H + OH
    {H2, OH, H2O, H, ELEM, 0},       //  2 H2 + OH = H2O + H
    {OH, OH, O, H2O, ELEM, 0},       //  3 OH + OH = O + H2O
    {H2, NONE, H, H, THIRD_BODY, 0}, //  4 H2 + M = H + H + M
    {O, O, O2, NONE, THIRD_BODY, 0}, //  5 O + O + M = O2 + M
    {O, H, OH, NONE, THIRD_BODY, 0}, //  6 O + H + M = OH + M
    {H, OH, H2O, NONE, THIRD_BODY, 0}, // 7 H + OH + M = H2O + M
    {H, O2, HO2, NONE, FALLOFF, 4},  //  8 H + O2 (+M) = HO2 (+M)
    {HO2, H, H2, O2, ELEM, 0},       //  9 HO2 + H = H2 + O2
    {HO2, H, OH, OH, ELEM, 0},       // 10 HO2 + H = OH + OH
    {HO2, O, O2, OH, ELEM, 0},       // 11 HO2 + O = O2 + OH
    {HO2, OH, H2O, O2, ELEM, 0},     // 12 HO2 + OH = H2O + O2
    {HO2, HO2, H2O2, O2, ELEM, 0},   // 13 HO2 + HO2 = H2O2 + O2 (duplicate)
    {HO2, HO2, H2O2, O2, ELEM, 0},   // 14 HO2 + HO2 = H2O2 + O2 (duplicate)
    {H2O2, NONE, OH, OH, FALLOFF, 3}, // 15 H2O2 (+M) = OH + OH (+M)
    {H2O2, H, H2O, OH, ELEM, 0},     // 16 H2O2 + H = H2O + OH
    {H2O2, H, HO2, H2, ELEM, 0},     // 17 H2O2 + H = HO2 + H2
    {H2O2, O, OH, HO2, ELEM, 0},     // 18 H2O2 + O = OH + HO2
    {H2O2, OH, HO2, H2O, ELEM, 0},   // 19 H2O2 + OH = HO2 + H2O (duplicate)
    {H2O2, OH, HO2, H2O, ELEM, 0},   // 20 H2O2 + OH = HO2 + H2O (duplicate)
};

__host__ __device__ constexpr int n_reac(const RxStruct &r) { return (r.r0 >= 0) + (r.r1 >= 0); }
__host__ __device__ constexpr int n_prod(const RxStruct &r) { return (r.p0 >= 0) + (r.p1 >= 0); }

// fp32 copies of the rate coefficients for the mixed-precision variant.
struct MechTablesF32 {
  float A[NRX];
  float W[NSP];
  float invW[NSP];
  float lnA[NRX], beta[NRX], Ta[NRX];
  float lnA0[NRX], beta0[NRX], Ta0[NRX];
  float troe_a[NRX], troe_i3[NRX], troe_i1[NRX], troe_T2[NRX];
  float effm1[NRX][NSP];
  // fp32 thermo for the surrogate's error test (all-fp32 right-hand side)
  float ec[2][NSP][6];
  float gc[2][NSP][7];
  float T_mid, ln_R_over_Pref;
  float newton_sq;  // the fp64 Newton's stop constant (below), tested in fp32
};

// Per-context tables (host-built from chem_mechanism by build_tables()).
struct MechTables {
  double T_mid;
  double W[NSP];
  double invW[NSP];
  // e_k W_k / R_u = sum_i ec[i] T^(i+1) + ec[5]: {a1 - 1, a2/2, a3/3, a4/4, a5/5, a6}
  double ec[2][NSP][6];
  // the same per unit mass fraction (ec / W_k): mixture coefficients sum_k Y_k ecw_k
  double ecw[2][NSP][6];
  // g_k / (R_u T) = h/RT - s/R = gc0 (1 - ln T) + gc1 T + gc2 T^2 + gc3 T^3 + gc4 T^4
  //                 + gc5 / T + gc6  with {a1, -a2/2, -a3/6, -a4/12, -a5/20, a6, -a7}
  double gc[2][NSP][7];
  // Arrhenius: k = exp(lnA + beta ln T - Ta / T); Ta = Ea / R_u.  kconst selects a form
  // without the exponential when Ea == 0: 1 for b == 0 (k = A), 2 for b == -1 (A / T),
  // 3 for b == -2 (A / T^2); 0 otherwise.
  double lnA[NRX], beta[NRX], Ta[NRX], A[NRX];
  int32_t kconst[NRX];
  int32_t reversible[NRX];
  // fall-off low-pressure limit and Troe parameters (alpha, 1/T***, 1/T*, T**)
  double lnA0[NRX], beta0[NRX], Ta0[NRX];
  double troe_a[NRX], troe_i3[NRX], troe_i1[NRX], troe_T2[NRX];
  // third-body efficiencies minus one: [M] = sum_k c_k + sum_k effm1 c_k
  double effm1[NRX][NSP];
  int32_t has_eff[NRX];
  int32_t eff_mask[NRX];  // bit k set where effm1[j][k] != 0 (the fp64 sums skip the rest)
  double ln_R_over_Pref;  // ln(R_u / p_ref): ln(R_u T / p_ref) = ln T + this
  // Newton's quadratic-convergence stop: after a step dT the remaining error is at most
  // (C / 2) dT^2 with C = max |c_v' / c_v| of the tables on [200, 6000] K, so a step with
  // dT^2 <= newton_sq T, newton_sq = 1e-12 / C, already leaves T within 1e-12 T / 2
  double newton_sq;
  // element mass fraction (H, O, N) per unit mass fraction of species k:
  // n_ke A_e / sum_e' n_ke' A_e' (columns sum to 1, so conserving elements conserves sum Y)
  double Emat[3][NSP];
  MechTablesF32 f;
};

static_assert(sizeof(MechTables) < 16384, "MechTables must fit a kernel parameter block");

}  // namespace chem

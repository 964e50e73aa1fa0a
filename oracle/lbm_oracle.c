/*
 * FP64 CPU oracle of the D3Q27 colour-fluid lattice Boltzmann update of
 * Saito, Abe & Koyama, "Lattice Boltzmann modeling and simulation of liquid
 * jet breakup" (arXiv 1705.03141), Sec. II, Sec. III and Sec. IV.A.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header or table with the CUDA library.
 *
 * It is written to be checked against the paper by eye, not to be fast:
 *   - dense 27x27 M and M^-1 typed from App. A (the printed matrices),
 *   - the collision done per colour exactly as Eq. (scoll) states it,
 *   - the enhanced equilibrium Eq. (EES) with phi_i^k (Eq. varphi_ik) and
 *     Phi_i^k (Eq. Phi), the MRT forcing of Eqs. (ketF)-(ketFd), the
 *     perturbation Eq. (perturb) and the recolouring of Sec. II,
 *   - pull streaming between two arrays.
 *
 * Readings of passages the paper leaves open (each listed in the design notes):
 *   R1  Eq. (perturb) is taken with the square restored: w_i (c_i.grad phi)^2/|grad phi|^2.
 *       The printed, unsquared form is kept behind `perturb_literal` so the
 *       tests can show that it breaks per-colour mass conservation.
 *       (Likewise `drop_Phi` removes the Phi term of Eq. (EES), so the tests
 *       can show what it does for a translating drop.)
 *   R3  the body force |F> enters once per node, split between the colours
 *       as (rho_k/rho)|F>.
 *   R5  cos(theta_1) = 0 for the rest vector.
 *   R6  where |grad phi|^2 <= 1e-24 the unit normal is taken as 0.
 *   R7  the LBE stores the full recoloured population (Omega^(3)).
 *   R10 gradients next to a non-periodic face use a mirror ghost value
 *       (the neighbour index is clamped into the box).
 *   R12 body force F = (rho - rho_ref) g with rho_ref = (rho_r0+rho_b0)/2
 *       (Rayleigh-Taylor) or rho_b0 (jet, Eq. bodyForceJet); a third mode
 *       applies a uniform force density F = g.
 *   R13 no-slip: halfway bounce-back; free-slip: specular reflection per
 *       wall-normal component.
 *   R14 the inlet is a layer of Dirichlet nodes on the z=0 plane inside the
 *       disk (x-xc)^2+(y-yc)^2 < (D/2)^2 that emit f^r = f^{r(e)}(rho_r0, u_in,
 *       alpha_r) with Phi = 0 and f^b = 0; the rest of that plane is a
 *       free-slip wall; optional uniform velocity noise from SplitMix64.
 *   R15 convective outflow on the z=nz-1 plane for every population of both
 *       colours, lambda = max(0, u_z(x, y, nz-2, t+1)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 27

/* Lattice velocities c_i, Eq. (velSet); their order is the one fixed by
 * rows 2-4 of the printed transformation matrix (App. A). */
static const int C[Q][3] = {
  { 0, 0, 0},
  { 1, 0, 0}, {-1, 0, 0}, { 0, 1, 0}, { 0,-1, 0}, { 0, 0, 1}, { 0, 0,-1},
  { 1, 1, 0}, {-1,-1, 0}, { 1,-1, 0}, {-1, 1, 0},
  { 0, 1, 1}, { 0,-1,-1}, { 0, 1,-1}, { 0,-1, 1},
  { 1, 0, 1}, {-1, 0,-1}, {-1, 0, 1}, { 1, 0,-1},
  { 1, 1, 1}, {-1,-1,-1}, { 1, 1,-1}, {-1,-1, 1},
  {-1, 1, 1}, { 1,-1,-1}, { 1,-1, 1}, {-1, 1,-1}};

/* Transformation matrix M, App. A (c = 1). */
static const double MM[Q][Q] = {
  {  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1,  1},
  {  0,  1, -1,  0,  0,  0,  0,  1, -1,  1, -1,  0,  0,  0,  0,  1, -1, -1,  1,  1, -1,  1, -1, -1,  1,  1, -1},
  {  0,  0,  0,  1, -1,  0,  0,  1, -1, -1,  1,  1, -1,  1, -1,  0,  0,  0,  0,  1, -1,  1, -1,  1, -1, -1,  1},
  {  0,  0,  0,  0,  0,  1, -1,  0,  0,  0,  0,  1, -1, -1,  1,  1, -1,  1, -1,  1, -1, -1,  1,  1, -1,  1, -1},
  { -2, -1, -1, -1, -1, -1, -1,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  1,  1,  1,  1,  1,  1,  1,  1},
  {  0,  2,  2, -1, -1, -1, -1,  1,  1,  1,  1, -2, -2, -2, -2,  1,  1,  1,  1,  0,  0,  0,  0,  0,  0,  0,  0},
  {  0,  0,  0,  1,  1, -1, -1,  1,  1,  1,  1,  0,  0,  0,  0, -1, -1, -1, -1,  0,  0,  0,  0,  0,  0,  0,  0},
  {  0,  0,  0,  0,  0,  0,  0,  1,  1, -1, -1,  0,  0,  0,  0,  0,  0,  0,  0,  1,  1,  1,  1, -1, -1, -1, -1},
  {  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  1,  1, -1, -1,  0,  0,  0,  0,  1,  1, -1, -1,  1,  1, -1, -1},
  {  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  1,  1, -1, -1,  1,  1, -1, -1, -1, -1,  1,  1},
  {  0, -4,  4,  0,  0,  0,  0, -1,  1, -1,  1,  0,  0,  0,  0, -1,  1,  1, -1,  2, -2,  2, -2, -2,  2,  2, -2},
  {  0,  0,  0, -4,  4,  0,  0, -1,  1,  1, -1, -1,  1, -1,  1,  0,  0,  0,  0,  2, -2,  2, -2,  2, -2, -2,  2},
  {  0,  0,  0,  0,  0, -4,  4,  0,  0,  0,  0, -1,  1,  1, -1, -1,  1, -1,  1,  2, -2, -2,  2,  2, -2,  2, -2},
  {  0,  4, -4,  0,  0,  0,  0, -2,  2, -2,  2,  0,  0,  0,  0, -2,  2,  2, -2,  1, -1,  1, -1, -1,  1,  1, -1},
  {  0,  0,  0,  4, -4,  0,  0, -2,  2,  2, -2, -2,  2, -2,  2,  0,  0,  0,  0,  1, -1,  1, -1,  1, -1, -1,  1},
  {  0,  0,  0,  0,  0,  4, -4,  0,  0,  0,  0, -2,  2,  2, -2, -2,  2, -2,  2,  1, -1, -1,  1,  1, -1,  1, -1},
  {  4,  0,  0,  0,  0,  0,  0, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,  1,  1,  1,  1,  1,  1,  1,  1},
  { -8,  4,  4,  4,  4,  4,  4, -2, -2, -2, -2, -2, -2, -2, -2, -2, -2, -2, -2,  1,  1,  1,  1,  1,  1,  1,  1},
  {  0, -4, -4,  2,  2,  2,  2,  1,  1,  1,  1, -2, -2, -2, -2,  1,  1,  1,  1,  0,  0,  0,  0,  0,  0,  0,  0},
  {  0,  0,  0, -2, -2,  2,  2,  1,  1,  1,  1,  0,  0,  0,  0, -1, -1, -1, -1,  0,  0,  0,  0,  0,  0,  0,  0},
  {  0,  0,  0,  0,  0,  0,  0, -2, -2,  2,  2,  0,  0,  0,  0,  0,  0,  0,  0,  1,  1,  1,  1, -1, -1, -1, -1},
  {  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0, -2, -2,  2,  2,  0,  0,  0,  0,  1,  1, -1, -1,  1,  1, -1, -1},
  {  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0, -2, -2,  2,  2,  1,  1, -1, -1, -1, -1,  1,  1},
  {  0,  0,  0,  0,  0,  0,  0,  1, -1,  1, -1,  0,  0,  0,  0, -1,  1,  1, -1,  0,  0,  0,  0,  0,  0,  0,  0},
  {  0,  0,  0,  0,  0,  0,  0, -1,  1,  1, -1,  1, -1,  1, -1,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0},
  {  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0, -1,  1,  1, -1,  1, -1,  1, -1,  0,  0,  0,  0,  0,  0,  0,  0},
  {  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  1, -1, -1,  1, -1,  1, -1,  1}
};

/* 216 M^-1, App. A. */
static const double MI216[Q][Q] = {
  {  8,  0,  0,  0,-24,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0,  0, 24, -8,  0,  0,  0,  0,  0,  0,  0,  0,  0},
  {  8, 12,  0,  0,-12, 12,  0,  0,  0,  0,-12,  0,  0, 12,  0,  0,  0,  4,-12,  0,  0,  0,  0,  0,  0,  0,  0},
  {  8,-12,  0,  0,-12, 12,  0,  0,  0,  0, 12,  0,  0,-12,  0,  0,  0,  4,-12,  0,  0,  0,  0,  0,  0,  0,  0},
  {  8,  0, 12,  0,-12, -6, 18,  0,  0,  0,  0,-12,  0,  0, 12,  0,  0,  4,  6,-18,  0,  0,  0,  0,  0,  0,  0},
  {  8,  0,-12,  0,-12, -6, 18,  0,  0,  0,  0, 12,  0,  0,-12,  0,  0,  4,  6,-18,  0,  0,  0,  0,  0,  0,  0},
  {  8,  0,  0, 12,-12, -6,-18,  0,  0,  0,  0,  0,-12,  0,  0, 12,  0,  4,  6, 18,  0,  0,  0,  0,  0,  0,  0},
  {  8,  0,  0,-12,-12, -6,-18,  0,  0,  0,  0,  0, 12,  0,  0,-12,  0,  4,  6, 18,  0,  0,  0,  0,  0,  0,  0},
  {  8, 12, 12,  0,  0,  6, 18, 18,  0,  0, -3, -3,  0, -6, -6,  0, -6, -2,  3,  9,-18,  0,  0, 27,-27,  0,  0},
  {  8,-12,-12,  0,  0,  6, 18, 18,  0,  0,  3,  3,  0,  6,  6,  0, -6, -2,  3,  9,-18,  0,  0,-27, 27,  0,  0},
  {  8, 12,-12,  0,  0,  6, 18,-18,  0,  0, -3,  3,  0, -6,  6,  0, -6, -2,  3,  9, 18,  0,  0, 27, 27,  0,  0},
  {  8,-12, 12,  0,  0,  6, 18,-18,  0,  0,  3, -3,  0,  6, -6,  0, -6, -2,  3,  9, 18,  0,  0,-27,-27,  0,  0},
  {  8,  0, 12, 12,  0,-12,  0,  0, 18,  0,  0, -3, -3,  0, -6, -6, -6, -2, -6,  0,  0,-18,  0,  0, 27,-27,  0},
  {  8,  0,-12,-12,  0,-12,  0,  0, 18,  0,  0,  3,  3,  0,  6,  6, -6, -2, -6,  0,  0,-18,  0,  0,-27, 27,  0},
  {  8,  0, 12,-12,  0,-12,  0,  0,-18,  0,  0, -3,  3,  0, -6,  6, -6, -2, -6,  0,  0, 18,  0,  0, 27, 27,  0},
  {  8,  0,-12, 12,  0,-12,  0,  0,-18,  0,  0,  3, -3,  0,  6, -6, -6, -2, -6,  0,  0, 18,  0,  0,-27,-27,  0},
  {  8, 12,  0, 12,  0,  6,-18,  0,  0, 18, -3,  0, -3, -6,  0, -6, -6, -2,  3, -9,  0,  0,-18,-27,  0, 27,  0},
  {  8,-12,  0,-12,  0,  6,-18,  0,  0, 18,  3,  0,  3,  6,  0,  6, -6, -2,  3, -9,  0,  0,-18, 27,  0,-27,  0},
  {  8,-12,  0, 12,  0,  6,-18,  0,  0,-18,  3,  0, -3,  6,  0, -6, -6, -2,  3, -9,  0,  0, 18, 27,  0, 27,  0},
  {  8, 12,  0,-12,  0,  6,-18,  0,  0,-18, -3,  0,  3, -6,  0,  6, -6, -2,  3, -9,  0,  0, 18,-27,  0,-27,  0},
  {  8, 12, 12, 12, 12,  0,  0, 18, 18, 18,  6,  6,  6,  3,  3,  3,  6,  1,  0,  0,  9,  9,  9,  0,  0,  0, 27},
  {  8,-12,-12,-12, 12,  0,  0, 18, 18, 18, -6, -6, -6, -3, -3, -3,  6,  1,  0,  0,  9,  9,  9,  0,  0,  0,-27},
  {  8, 12, 12,-12, 12,  0,  0, 18,-18,-18,  6,  6, -6,  3,  3, -3,  6,  1,  0,  0,  9, -9, -9,  0,  0,  0,-27},
  {  8,-12,-12, 12, 12,  0,  0, 18,-18,-18, -6, -6,  6, -3, -3,  3,  6,  1,  0,  0,  9, -9, -9,  0,  0,  0, 27},
  {  8,-12, 12, 12, 12,  0,  0,-18, 18,-18, -6,  6,  6, -3,  3,  3,  6,  1,  0,  0, -9,  9, -9,  0,  0,  0,-27},
  {  8, 12,-12,-12, 12,  0,  0,-18, 18,-18,  6, -6, -6,  3, -3, -3,  6,  1,  0,  0, -9,  9, -9,  0,  0,  0, 27},
  {  8, 12,-12, 12, 12,  0,  0,-18,-18, 18,  6, -6,  6,  3, -3,  3,  6,  1,  0,  0, -9, -9,  9,  0,  0,  0,-27},
  {  8,-12, 12,-12, 12,  0,  0,-18,-18, 18, -6,  6, -6, -3,  3, -3,  6,  1,  0,  0, -9, -9,  9,  0,  0,  0, 27}
};

/* Relaxation-rate slot of each moment: K = diag[s1,s1,s1,s1,s5,s6,s6,s8,s8,s8,
 * s11,s11,s11,s14,s14,s14,s17,s18,s19,s19,s21,s21,s21,s24,s24,s24,s27]
 * (Sec. II, equation for K). Values are 1-based rate indices. */
static const int KSLOT[Q] = {1,1,1,1,5,6,6,8,8,8,11,11,11,14,14,14,17,18,19,19,21,21,21,24,24,24,27};

/* velocity group: 0 rest, 1 axis (i=2..7), 2 edge (8..19), 3 corner (20..27) */
static int group_of(int i) { return i == 0 ? 0 : (i < 7 ? 1 : (i < 19 ? 2 : 3)); }

/* w_i, Sec. II (D3Q27 weights). */
static double weight(int i) {
  static const double wg[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
  return wg[group_of(i)];
}
/* varphi_i^k, Eq. (varphi_ik). */
static double varphi(int i, double alpha) {
  switch (group_of(i)) {
    case 0: return alpha;
    case 1: return 2.0 * (1.0 - alpha) / 19.0;
    case 2: return (1.0 - alpha) / 38.0;
    default: return (1.0 - alpha) / 152.0;
  }
}
/* B_i, Eq. (B_i) with c = 1. */
static double Bcoef(int i) {
  static const double bg[4] = {-10.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
  return bg[group_of(i)];
}
/* leading factor of Phi_i^k, Eq. (Phi): -3 for i=1, 16/4/1 by group. */
static double phi_factor(int i) {
  static const double ag[4] = {-3.0, 16.0, 4.0, 1.0};
  return ag[group_of(i)];
}
static int opposite(int i) { return i == 0 ? 0 : (i % 2 == 1 ? i + 1 : i - 1); }

enum { BC_PERIODIC = 0, BC_NOSLIP = 1, BC_FREESLIP = 2, BC_INFLOW_WALL = 3, BC_OUTFLOW = 4 };

typedef struct {
  double rho_r0, rho_b0;   /* initial phase densities; gamma = rho_r0/rho_b0 */
  double nu_r, nu_b;       /* kinematic viscosities */
  double A, beta;          /* perturbation strength, recolouring parameter */
  double s[Q];             /* s[j-1] = rate s_j; s6 and s8 are replaced per node */
  double g[3];             /* gravity / force vector */
  int force_mode;          /* 0 none, 1 (rho - (rho_r0+rho_b0)/2) g, 2 (rho - rho_b0) g, 3 g */
  int bc[6];               /* -x,+x,-y,+y,-z,+z */
  int inflow;              /* 1: Dirichlet inlet disk on the z=0 plane (needs bc[4]==INFLOW_WALL) */
  double xc, yc, D, u_j0, noise_frac;
  uint64_t seed;
  int perturb_literal;     /* 1: Eq. (perturb) exactly as printed (no square) */
  int ghost_mode;          /* gradient ghost next to a wall: 0 mirror (R10); 1 periodic wrap and
                              2 mirror about the wall node are planted mistakes for the tests */
  int drop_Phi;            /* 1: Phi_i^k = 0 in the collision (a planted mistake for the tests) */
} orc_params;

/* alpha_b = 8/27 (Sec. II); Grunau relation gamma = (1-alpha_b)/(1-alpha_r). */
static double alpha_b(void) { return 8.0 / 27.0; }
static double alpha_r(const orc_params* p) {
  double gamma = p->rho_r0 / p->rho_b0;
  return 1.0 - (1.0 - alpha_b()) / gamma;
}

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): counter-based hash used for
 * the seeded inlet noise; xi in [-1, 1) from the top 53 bits. */
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
double orc_noise(uint64_t seed, int64_t t, int64_t node, int comp) {
  uint64_t h = splitmix64(seed);
  h = splitmix64(h ^ (uint64_t)t);
  h = splitmix64(h ^ (uint64_t)node);
  h = splitmix64(h ^ (uint64_t)comp);
  return (double)(h >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
}

/* ------------------------------------------------------------------ */
/* tables for the tests                                                */
void orc_tables(int* c, double* M, double* Minv, double* w, double* B, int* kslot) {
  for (int i = 0; i < Q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = C[i][a];
    w[i] = weight(i);
    B[i] = Bcoef(i);
    kslot[i] = KSLOT[i];
    for (int j = 0; j < Q; ++j) {
      M[Q * i + j] = MM[i][j];
      Minv[Q * i + j] = MI216[i][j] / 216.0;
    }
  }
}
double orc_varphi(int i, double alpha) { return varphi(i, alpha); }
double orc_alpha_r(const orc_params* p) { return alpha_r(p); }

/* Phi_i (Eq. Phi) for one colour: nubar, u, grad rho_k. */
void orc_Phi(double nubar, const double* u, const double* grad, double* out) {
  double G[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) G[a][b] = (u[a] * grad[b] + u[b] * grad[a]) / 48.0;
  for (int i = 0; i < Q; ++i) {
    if (i == 0) {
      out[i] = phi_factor(0) * nubar * (u[0] * grad[0] + u[1] * grad[1] + u[2] * grad[2]);
    } else {
      double gcc = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) gcc += G[a][b] * C[i][a] * C[i][b];
      out[i] = phi_factor(i) * nubar * gcc;
    }
  }
}

/* f_i^{k(e)}(rho_k, u, alpha_k) + Phi_i^k, Eq. (EES). */
static void equilibrium(double rho_k, const double* u, double alpha, const double* Phi, double* out) {
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < Q; ++i) {
    double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
    out[i] = rho_k * (varphi(i, alpha) + weight(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu)) + (Phi ? Phi[i] : 0.0);
  }
}
void orc_equilibrium(double rho_k, const double* u, double alpha, const double* Phi, double* out) {
  equilibrium(rho_k, u, alpha, Phi, out);
}

/* y = A x for a dense 27x27 matrix */
static void matvec(const double A[Q][Q], double scale, const double* x, double* y) {
  for (int i = 0; i < Q; ++i) {
    double s = 0.0;
    for (int j = 0; j < Q; ++j) s += A[i][j] * x[j];
    y[i] = s * scale;
  }
}

/* ------------------------------------------------------------------ */
/* geometry                                                            */
typedef struct { int nx, ny, nz; } dims;
static int64_t lin(const dims* d, int x, int y, int z) { return (int64_t)x + (int64_t)d->nx * ((int64_t)y + (int64_t)d->ny * z); }

static int is_inlet(const orc_params* p, const dims* d, int x, int y, int z) {
  (void)d;
  if (!p->inflow || z != 0) return 0;
  double dx = x - p->xc, dy = y - p->yc;
  return dx * dx + dy * dy < 0.25 * p->D * p->D;
}

/* neighbour used by the gradient stencil: periodic wrap, otherwise the mirror ghost of R10
 * (the index is clamped into the box: the ghost one link outside a wall carries the value of
 * the wall node, a mirror about the half-link plane where the walls reflect).  ghost_mode 1
 * and 2 are deliberately wrong readings (wrap across a wall; mirror about the wall node) that
 * only the tests select, to show that the wall-symmetry pin detects them. */
static int nb_coord(int q, int n, int bc_lo, int bc_hi, int ghost_mode) {
  if (q < 0) {
    if (bc_lo == BC_PERIODIC || ghost_mode == 1) return q + n;
    return ghost_mode == 2 ? -q : 0;
  }
  if (q >= n) {
    if (bc_hi == BC_PERIODIC || ghost_mode == 1) return q - n;
    return ghost_mode == 2 ? 2 * (n - 1) - q : n - 1;
  }
  return q;
}

/* Where does the population leaving node (x,y,z) along c_i arrive?
 * Periodic faces wrap; free-slip and inflow-wall faces reflect the
 * wall-normal component (the node coordinate stays); a no-slip face
 * returns it to the same node reversed (halfway bounce-back); an outflow
 * face lets it leave (returns 0).  Returns 1 with (*ox,*oy,*oz,*oi). */
static int push_target(const orc_params* p, const dims* d, int x, int y, int z, int i,
                       int* ox, int* oy, int* oz, int* oi) {
  int pos[3] = {x, y, z}, n[3] = {d->nx, d->ny, d->nz};
  int cv[3] = {C[i][0], C[i][1], C[i][2]};
  int out[3], bounce = 0, leaves = 0;
  for (int a = 0; a < 3; ++a) {
    int q = pos[a] + cv[a];
    out[a] = q;
    if (q >= 0 && q < n[a]) continue;
    int bc = q < 0 ? p->bc[2 * a] : p->bc[2 * a + 1];
    if (bc == BC_PERIODIC) out[a] = q < 0 ? q + n[a] : q - n[a];
    else if (bc == BC_NOSLIP) bounce = 1;
    else if (bc == BC_OUTFLOW) leaves = 1;
    else { out[a] = pos[a]; cv[a] = -cv[a]; }       /* specular */
  }
  if (bounce) { *ox = x; *oy = y; *oz = z; *oi = opposite(i); return 1; }
  if (leaves) return 0;
  int j;
  for (j = 0; j < Q; ++j)
    if (C[j][0] == cv[0] && C[j][1] == cv[1] && C[j][2] == cv[2]) break;
  *ox = out[0]; *oy = out[1]; *oz = out[2]; *oi = j;
  return 1;
}

/* ------------------------------------------------------------------ */
/* one node: collision + perturbation + recolouring                    */
typedef struct {
  const double *rr, *rb;   /* rho_r, rho_b fields used by the gradient (Eq. for grad chi) */
} fields;

static void node_update(const orc_params* p, const dims* d, const double* f, const fields* fl,
                        int x, int y, int z, int64_t t, double* outr, double* outb) {
  const int64_t N = (int64_t)d->nx * d->ny * d->nz;
  const int64_t n0 = lin(d, x, y, z);
  const double ar = alpha_r(p), ab = alpha_b();

  if (is_inlet(p, d, x, y, z)) {
    /* R14: Dirichlet equilibrium of the dispersed phase at the inlet. */
    double u[3] = {0.0, 0.0, p->u_j0};
    if (p->noise_frac != 0.0)
      for (int a = 0; a < 3; ++a) u[a] += p->u_j0 * p->noise_frac * orc_noise(p->seed, t, n0, a);
    equilibrium(p->rho_r0, u, ar, NULL, outr);
    for (int i = 0; i < Q; ++i) outb[i] = 0.0;
    return;
  }

  double fr[Q], fb[Q];
  for (int i = 0; i < Q; ++i) { fr[i] = f[(int64_t)i * N + n0]; fb[i] = f[(int64_t)(Q + i) * N + n0]; }

  /* densities (Sec. II) and order parameter, Eq. (order) */
  double rho_r = 0.0, rho_b = 0.0;
  for (int i = 0; i < Q; ++i) { rho_r += fr[i]; rho_b += fb[i]; }
  double rho = rho_r + rho_b;
  double phi = (rho_r - rho_b) / rho;

  /* isotropic central gradients of phi, rho_r, rho_b (Sec. II, gradient scheme) */
  double gphi[3] = {0, 0, 0}, grr[3] = {0, 0, 0}, grb[3] = {0, 0, 0};
  for (int i = 1; i < Q; ++i) {
    int xx = nb_coord(x + C[i][0], d->nx, p->bc[0], p->bc[1], p->ghost_mode);
    int yy = nb_coord(y + C[i][1], d->ny, p->bc[2], p->bc[3], p->ghost_mode);
    int zz = nb_coord(z + C[i][2], d->nz, p->bc[4], p->bc[5], p->ghost_mode);
    int64_t m = lin(d, xx, yy, zz);
    double r = fl->rr[m], b = fl->rb[m];
    double ph = (r - b) / (r + b);
    for (int a = 0; a < 3; ++a) {
      gphi[a] += 3.0 * weight(i) * ph * C[i][a];
      grr[a] += 3.0 * weight(i) * r * C[i][a];
      grb[a] += 3.0 * weight(i) * b * C[i][a];
    }
  }

  /* body force (R12) and velocity with the half-force shift, Eq. (Momentum) */
  double F[3] = {0, 0, 0};
  if (p->force_mode == 1 || p->force_mode == 2) {
    double ref = p->force_mode == 1 ? 0.5 * (p->rho_r0 + p->rho_b0) : p->rho_b0;
    for (int a = 0; a < 3; ++a) F[a] = (rho - ref) * p->g[a];
  } else if (p->force_mode == 3) {
    for (int a = 0; a < 3; ++a) F[a] = p->g[a];
  }
  double u[3];
  for (int a = 0; a < 3; ++a) {
    double mom = 0.0;
    for (int i = 0; i < Q; ++i) mom += (fr[i] + fb[i]) * C[i][a];
    u[a] = (mom + 0.5 * F[a]) / rho;
  }

  /* interpolated viscosity and the shear rates s6 = s8, Eq. (shear) */
  double nubar = 0.5 * (1.0 + phi) * p->nu_r + 0.5 * (1.0 - phi) * p->nu_b;
  double s_shear = 1.0 / (3.0 * nubar + 0.5);
  double K[Q];
  for (int j = 0; j < Q; ++j) {
    int slot = KSLOT[j];
    K[j] = (slot == 6 || slot == 8) ? s_shear : p->s[slot - 1];
  }

  /* MRT forcing |F> = M^-1 (I - K/2) M |F'>, Eqs. (ketF)-(ketFd) */
  double Fp[Q], mF[Q], Fket[Q];
  for (int i = 0; i < Q; ++i) {
    double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
    double acc = 0.0;
    for (int a = 0; a < 3; ++a) acc += (3.0 * (C[i][a] - u[a]) + 9.0 * cu * C[i][a]) * F[a];
    Fp[i] = weight(i) * acc;
  }
  matvec(MM, 1.0, Fp, mF);
  for (int j = 0; j < Q; ++j) mF[j] *= (1.0 - 0.5 * K[j]);
  matvec(MI216, 1.0 / 216.0, mF, Fket);

  /* perturbation operator, Eq. (perturb) (R1: square restored) */
  double g2 = gphi[0] * gphi[0] + gphi[1] * gphi[1] + gphi[2] * gphi[2];
  double gnorm = sqrt(g2);
  int has_normal = g2 > 1e-24;

  double post[2][Q];
  for (int k = 0; k < 2; ++k) {
    const double* fk = k == 0 ? fr : fb;
    double rho_k = k == 0 ? rho_r : rho_b;
    double alpha_k = k == 0 ? ar : ab;
    const double* gk = k == 0 ? grr : grb;
    double Phi[Q], feq[Q], neq[Q], m[Q], coll[Q];
    orc_Phi(nubar, u, gk, Phi);
    if (p->drop_Phi) memset(Phi, 0, sizeof Phi);
    equilibrium(rho_k, u, alpha_k, Phi, feq);
    for (int i = 0; i < Q; ++i) neq[i] = fk[i] - feq[i];
    matvec(MM, 1.0, neq, m);
    for (int j = 0; j < Q; ++j) m[j] *= K[j];
    matvec(MI216, 1.0 / 216.0, m, coll);
    for (int i = 0; i < Q; ++i) {
      double om2 = 0.0;
      if (has_normal) {
        double cg = C[i][0] * gphi[0] + C[i][1] * gphi[1] + C[i][2] * gphi[2];
        double shape = p->perturb_literal ? weight(i) * cg / g2 : weight(i) * cg * cg / g2;
        om2 = 0.5 * p->A * gnorm * (shape - Bcoef(i));
      }
      post[k][i] = fk[i] - coll[i] + (rho_k / rho) * Fket[i] + om2;
    }
  }

  /* recolouring operator Omega^(3) (Sec. II) with f^(e)(rho, 0, alpha_bar) = rho varphi_i(alpha_bar) */
  double abar = 0.5 * (1.0 + phi) * ar + 0.5 * (1.0 - phi) * ab;
  double coef = p->beta * rho_r * rho_b / (rho * rho);
  for (int i = 0; i < Q; ++i) {
    double fstar = post[0][i] + post[1][i];
    double cos_t = 0.0;
    if (i != 0 && has_normal) {
      double cn = sqrt((double)(C[i][0] * C[i][0] + C[i][1] * C[i][1] + C[i][2] * C[i][2]));
      cos_t = (C[i][0] * gphi[0] + C[i][1] * gphi[1] + C[i][2] * gphi[2]) / (cn * gnorm);
    }
    double feq0 = rho * varphi(i, abar);
    outr[i] = (rho_r / rho) * fstar + coef * cos_t * feq0;
    outb[i] = (rho_b / rho) * fstar - coef * cos_t * feq0;
  }
}

/* ------------------------------------------------------------------ */
/* one time step over the whole box                                   */
/* f: [2][27][nz][ny][nx] in/out; top: [2][27][ny][nx] saved outflow plane (R15), may be NULL */
int orc_step(const orc_params* p, int nx, int ny, int nz, int64_t t, double* f, double* top) {
  dims d = {nx, ny, nz};
  const int64_t N = (int64_t)nx * ny * nz;
  double* rr = (double*)malloc(sizeof(double) * N);
  double* rb = (double*)malloc(sizeof(double) * N);
  double* post = (double*)malloc(sizeof(double) * 2 * Q * N);
  if (!rr || !rb || !post) { free(rr); free(rb); free(post); return -2; }

  /* phase densities; inlet nodes carry the prescribed rho_r0 / 0 (R14) */
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t n0 = lin(&d, x, y, z);
        double r = 0.0, b = 0.0;
        for (int i = 0; i < Q; ++i) { r += f[(int64_t)i * N + n0]; b += f[(int64_t)(Q + i) * N + n0]; }
        if (is_inlet(p, &d, x, y, z)) { r = p->rho_r0; b = 0.0; }
        rr[n0] = r; rb[n0] = b;
      }

  fields fl = {rr, rb};
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t n0 = lin(&d, x, y, z);
        double outr[Q], outb[Q];
        node_update(p, &d, f, &fl, x, y, z, t, outr, outb);
        for (int i = 0; i < Q; ++i) { post[(int64_t)i * N + n0] = outr[i]; post[(int64_t)(Q + i) * N + n0] = outb[i]; }
      }

  /* streaming, Eq. (LBE): push every post-collision value to its target */
  for (int64_t q = 0; q < 2 * Q * N; ++q) f[q] = 0.0;
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x)
        for (int i = 0; i < Q; ++i) {
          int ox, oy, oz, oi;
          if (!push_target(p, &d, x, y, z, i, &ox, &oy, &oz, &oi)) continue;
          int64_t src = lin(&d, x, y, z), dst = lin(&d, ox, oy, oz);
          f[(int64_t)oi * N + dst] = post[(int64_t)i * N + src];
          f[(int64_t)(Q + oi) * N + dst] = post[(int64_t)(Q + i) * N + src];
        }

  /* convective outflow, Sec. IV.A (R15) */
  if (p->bc[5] == BC_OUTFLOW && top) {
    const int64_t P = (int64_t)nx * ny;
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int64_t nN = lin(&d, x, y, nz - 1), nM = lin(&d, x, y, nz - 2);
        double rho = 0.0, mz = 0.0;
        for (int i = 0; i < Q; ++i) {
          double fi = f[(int64_t)i * N + nM] + f[(int64_t)(Q + i) * N + nM];
          rho += fi; mz += fi * C[i][2];
        }
        double Fz = 0.0;
        if (p->force_mode == 1) Fz = (rho - 0.5 * (p->rho_r0 + p->rho_b0)) * p->g[2];
        else if (p->force_mode == 2) Fz = (rho - p->rho_b0) * p->g[2];
        else if (p->force_mode == 3) Fz = p->g[2];
        double uz = (mz + 0.5 * Fz) / rho;
        double lam = uz > 0.0 ? uz : 0.0;
        int64_t pp = lin(&d, x, y, 0);
        for (int k = 0; k < 2; ++k)
          for (int i = 0; i < Q; ++i) {
            int64_t s = (int64_t)(k * Q + i);
            double fn = (top[s * P + pp] + lam * f[s * N + nM]) / (1.0 + lam);
            f[s * N + nN] = fn;
            top[s * P + pp] = fn;
          }
      }
  }
  free(rr); free(rb); free(post);
  return 0;
}

int orc_run(const orc_params* p, int nx, int ny, int nz, int64_t t0, int nsteps, double* f, double* top) {
  for (int s = 0; s < nsteps; ++s) {
    int rc = orc_step(p, nx, ny, nz, t0 + s, f, top);
    if (rc) return rc;
  }
  return 0;
}

/* initial populations f^k = f^{k(e)}(rho_k, u, alpha_k) with Phi = 0 (R9) */
void orc_init(const orc_params* p, int nx, int ny, int nz, const double* rr, const double* rb,
              const double* u /* [3][N] or NULL */, double* f) {
  const int64_t N = (int64_t)nx * ny * nz;
  const double ar = alpha_r(p), ab = alpha_b();
  for (int64_t n = 0; n < N; ++n) {
    double uu[3] = {0, 0, 0}, er[Q], eb[Q];
    if (u) { uu[0] = u[n]; uu[1] = u[N + n]; uu[2] = u[2 * N + n]; }
    equilibrium(rr[n], uu, ar, NULL, er);
    equilibrium(rb[n], uu, ab, NULL, eb);
    for (int i = 0; i < Q; ++i) { f[(int64_t)i * N + n] = er[i]; f[(int64_t)(Q + i) * N + n] = eb[i]; }
  }
}

/* macroscopic fields: rho_r, rho_b and u (Eq. Momentum, with the same force as the step) */
void orc_macro(const orc_params* p, int nx, int ny, int nz, const double* f, double* rr, double* rb, double* u) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t n = 0; n < N; ++n) {
    double r = 0.0, b = 0.0, m[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
      double a = f[(int64_t)i * N + n], c = f[(int64_t)(Q + i) * N + n];
      r += a; b += c;
      for (int k = 0; k < 3; ++k) m[k] += (a + c) * C[i][k];
    }
    double rho = r + b, F[3] = {0, 0, 0};
    if (p->force_mode == 1 || p->force_mode == 2) {
      double ref = p->force_mode == 1 ? 0.5 * (p->rho_r0 + p->rho_b0) : p->rho_b0;
      for (int k = 0; k < 3; ++k) F[k] = (rho - ref) * p->g[k];
    } else if (p->force_mode == 3) {
      for (int k = 0; k < 3; ++k) F[k] = p->g[k];
    }
    rr[n] = r; rb[n] = b;
    if (u) for (int k = 0; k < 3; ++k) u[(int64_t)k * N + n] = (m[k] + 0.5 * F[k]) / rho;
  }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

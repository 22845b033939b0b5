// Oracle for the RAPRAL hot path -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow FP64 CPU restatement of what the paper computes, written
// step by step in the paper's order and notation, with no blocking, fusion or
// reordering beyond what the method itself states.  Only the test suite, the
// package's smoke check and the benchmark's CPU-baseline leg may load it; the
// product path never does.  It shares no code with the CUDA library.
//
// Physics followed (RAPRAL, arXiv 2604.11856):
//   Sec. 2.1    Boltzmann electronic populations of atoms; molecular electronic
//               Boltzmann populations with the rovibrational partition function
//               Q_vr; rovibronic level populations (with S_multi / sigma).
//   Sec. 2.2    Planck function in temperature form and in population form.
//   Sec. 2.2.1  bound-bound emission j and absorption kappa = j / B; Whiting's
//               Voigt line shape; Voigt HWHM; Doppler HWHM; Lorentz HWHM as the
//               sum of natural and Stark widths; Stark width scaling.
//   Sec. 2.2.2  molecular bound-bound emission (same form as atoms).
//   Sec. 2.2.3  formal RTE solution marched segment by segment with kappa held
//               at the far node and j linear (the Johnston-Mazaheri scheme),
//               its thin-segment series, and the wall heat flux as a solid-angle
//               and wavelength integral.
//
// Readings taken where the paper is silent or inconsistent (all listed in the
// design notes): cgs constants as printed, results converted erg -> W by 1e-7;
// line wings cut at |dlam| <= 100 lamV (+-50 Voigt FWHM); Lorentz width =
// natural + Stark; T_ee = T_v = T_ve and T_r = T_tr; node values of a ray are
// the mean of the two cells adjacent to a face (one cell at the ends); the
// far/near coefficients of a segment are the ones that the paper's own
// integral of the linear emission gives; the thin-segment branch is a
// three-term series of both coefficients for |dtau| below a threshold.
//
// Summation over lines is Neumaier-compensated.  Compile with
// -ffp-contract=off so that x86 and Arm builds round identically.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// ---------------------------------------------------------------- inputs ----

typedef struct {
    int32_t S;                 // radiating species
    const int32_t* kind;       // [S] 0 atom, 1 diatomic molecule
    const int32_t* dens_col;   // [S] column of the species in the cell densities
    const double* mass;        // [S] molar mass, g/mol
    const int64_t* atom_off;   // [S+1] atomic level ranges
    const double* atom_E;      // level energy, cm^-1
    const double* atom_g;      // level degeneracy
    const int64_t* st_off;     // [S+1] molecular electronic-state ranges
    const double* st_E;        // electronic term energy, cm^-1
    const double* st_g;        // electronic degeneracy
    const double* st_sigma;    // symmetry factor
    const double* st_Lalt;     // [n_st*2] line alternation factor, even / odd J
    const int32_t* st_nv;      // vibrational levels per state
    const int32_t* st_nj;      // rotational levels per vibrational level
    const int64_t* st_vib_off; // offset into vib_E
    const int64_t* st_rot_off; // offset into rot_E ([V][J] per state)
    const double* vib_E;       // E_V, cm^-1
    const double* rot_E;       // E_J(V), cm^-1
} orc_species;

typedef struct {
    int64_t L;
    const double* lam0;   // nm
    const double* A;      // s^-1
    const double* lamS0;  // nm
    const int32_t* species;
    const double *Eu_el, *Eu_v, *Eu_j, *gu;
    const double *El_el, *El_v, *El_j, *gl;
} orc_lines;

typedef struct {
    int64_t C;
    const double* Ttr;
    const double* Tve;
    const double* n;      // [C*ncol]
    int32_t ncol;
    int32_t ne_col;
} orc_cells;

typedef struct {
    double lam_min, lam_max;
    int64_t n;
} orc_grid;

// ------------------------------------------------------------- constants ----
// Sec. 2.1 prints k, c and h in cgs with four digits; those are the default.

static double kB = 1.380e-16;   // erg/K
static double cL = 2.998e10;    // cm/s
static double hP = 6.626e-27;   // erg s

static double me_g = 9.109e-28, e_esu = 4.803e-10;   // electron mass (g) and charge (esu)

void orc_set_codata(int on) {
    if (on) { kB = 1.380649e-16; cL = 2.99792458e10; hP = 6.62607015e-27; me_g = 9.1093837e-28; e_esu = 4.80320471e-10; }
    else    { kB = 1.380e-16;    cL = 2.998e10;      hP = 6.626e-27;      me_g = 9.109e-28;     e_esu = 4.803e-10; }
}
double orc_c2(void) { return hP * cL / kB; }   // second radiation constant, cm K
double orc_const(int which) { return which == 0 ? kB : which == 1 ? cL : hP; }

// --------------------------------------------------------- populations ----

// Sec. 2.1, atomic Boltzmann distribution: denominator sum_j g_j exp(-hcE_j/kT_ee).
// Sec. 2.1, molecular Boltzmann distribution: sum_i g_i exp(-hcE_i/kT_ee) Q_vr,i with
//   Q_vr,i = sum_V exp(-hcE_V/kT_v) (1/sigma) sum_J (2J+1) L_alter exp(-hcE_J/kT_r).
// T_ee = T_v = T_ve, T_r = T_tr.
double orc_partition(const orc_species* sp, int32_t s, double Ttr, double Tve) {
    const double c2 = orc_c2();
    double Z = 0.0;
    if (sp->kind[s] == 0) {
        for (int64_t l = sp->atom_off[s]; l < sp->atom_off[s + 1]; ++l)
            Z += sp->atom_g[l] * std::exp(-c2 * sp->atom_E[l] / Tve);
        return Z;
    }
    for (int64_t i = sp->st_off[s]; i < sp->st_off[s + 1]; ++i) {
        double Qvr = 0.0;
        const int nv = sp->st_nv[i], nj = sp->st_nj[i];
        for (int v = 0; v < nv; ++v) {
            double rot = 0.0;
            for (int J = 0; J < nj; ++J) {
                const double EJ = sp->rot_E[sp->st_rot_off[i] + (int64_t)v * nj + J];
                rot += (2.0 * J + 1.0) * sp->st_Lalt[2 * i + (J & 1)] * std::exp(-c2 * EJ / Ttr);
            }
            Qvr += std::exp(-c2 * sp->vib_E[sp->st_vib_off[i] + v] / Tve) * rot / sp->st_sigma[i];
        }
        Z += sp->st_g[i] * std::exp(-c2 * sp->st_E[i] / Tve) * Qvr;
    }
    return Z;
}

// ln N_s - ln Z_s per cell and radiating species, [C][S].
void orc_lnpref(const orc_species* sp, const orc_cells* cells, double* lnpref) {
    const int64_t C = cells->C;
    const int S = sp->S;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < C; ++c)
        for (int s = 0; s < S; ++s) {
            const double N = cells->n[c * cells->ncol + sp->dens_col[s]];
            // a species with no particles has no population (ln 0 = -inf)
            if (!(N > 0.0)) { lnpref[c * S + s] = -INFINITY; continue; }
            const double Z = orc_partition(sp, s, cells->Ttr[c], cells->Tve[c]);
            lnpref[c * S + s] = std::log(N) - std::log(Z);
        }
}

// Sec. 2.1: level population N = (N_s / Z_s) g exp(-hc(E_el + E_V)/kT_ve - hcE_J/kT_tr),
// where g carries g_i S_multi (2J+1) L_alter / sigma for a rovibronic level.
double orc_ln_level_pop(double lnpref, double g, double E_el, double E_v, double E_j,
                        double Tve, double Ttr) {
    const double c2 = orc_c2();
    return lnpref + std::log(g) - c2 * (E_el / Tve + E_v / Tve + E_j / Ttr);
}

// ------------------------------------------------------------ spectroscopy ----

// Sec. 2.2: Planck function, temperature form, W/cm^2/sr/um (erg -> W: 1e-7).
double orc_planck(double lam_nm, double T) {
    const double lcm = lam_nm * 1e-7;
    const double x = hP * cL / (lcm * kB * T);
    return 1e-7 * 2.0 * hP * cL * cL / (1e4 * std::pow(lcm, 5) * std::expm1(x));
}

// Sec. 2.2.1: Doppler HWHM, lamG = (7.16233e-7 / 2) lam (T_t / M)^0.5.
double orc_doppler_hwhm(double lam0, double Ttr, double M) {
    return 7.16233e-7 / 2.0 * lam0 * std::sqrt(Ttr / M);
}
// Sec. 2.2.1: Stark HWHM, lamS = lamS0 (T_ee/1e4)^0.33 (N_e/1e16).
double orc_stark_hwhm(double lamS0, double Tve, double ne) {
    return lamS0 * std::pow(Tve / 10000.0, 0.33) * (ne / 1e16);
}
// Sec. 2.2.1: natural broadening constant.
static const double LAM_N = 5.9e-6;
// Sec. 2.2.1: Lorentz HWHM = natural + Stark (+ resonance + van der Waals when
// orc_set_broadening turns them on).
double orc_lorentz_hwhm(double lamS) { return LAM_N + lamS; }

// Sec. 2.2.1 full Lorentz broadening, off by default (flags 0):
//   1: Stark coefficient of atomic lines from the ionisation gap,
//      lamS0 = 1.69e3 lam^2 / dE^2.623, dE = max(E_ionize - E_u, E_ionize^H / 25);
//   2: resonance broadening of atomic lines whose lower level is the ground
//      level, lamR = 4.3e-28 lam f_lu N_0 (g_l/g_u)^0.5 lam^2 with the
//      oscillator strength f_lu = m_e c (lam 1e-7)^2 g_u A / (8 pi^2 e^2 g_l)
//      and N_0 the species' ground-level density;
//   4: van der Waals broadening of atomic lines,
//      lamW = lam^2 [6.65e-29 N (2 T_t/M)^0.5 + 2.925e-29 N_o (2 T_t/M_o)^0.5],
//      N, M the radiating species' density and molar mass, N_o the summed
//      density of the other heavy particles (every density column but the
//      species' own and those of molar mass 0, the electrons) and M_o their
//      density-weighted mean molar mass.
static int BROAD_FLAGS = 0;
static double BROAD_EION[64];      // per radiating species, cm^-1
static int BROAD_NCOL = 0;
static double BROAD_COLMASS[64];   // per density column, g/mol (0: electrons)
static const double E_IONIZE_H = 109678.77;   // cm^-1

void orc_set_broadening(int flags, int S, const double* E_ion, int ncol, const double* col_mass) {
    BROAD_FLAGS = flags;
    for (int s = 0; s < S && s < 64; ++s) BROAD_EION[s] = E_ion ? E_ion[s] : 0.0;
    BROAD_NCOL = ncol < 64 ? ncol : 64;
    for (int c = 0; c < BROAD_NCOL; ++c) BROAD_COLMASS[c] = col_mass ? col_mass[c] : 0.0;
}
double orc_stark_coeff_ionize(double lam0, double Eu, double Eion) {
    const double dE = std::max(Eion - Eu, E_IONIZE_H / 25.0);
    return 1.69e3 * lam0 * lam0 / std::pow(dE, 2.623);
}
double orc_oscillator_strength(double lam0, double A, double gu, double gl) {
    const double lcm = lam0 * 1e-7;
    return me_g * cL * lcm * lcm / (8.0 * M_PI * M_PI * e_esu * e_esu) * gu / gl * A;
}
double orc_resonance_hwhm(double lam0, double A, double gu, double gl, double N0) {
    const double f = orc_oscillator_strength(lam0, A, gu, gl);
    return 4.3e-28 * lam0 * f * N0 * std::sqrt(gl / gu) * lam0 * lam0;
}
double orc_vdw_hwhm(double lam0, double Ttr, double N, double M, double No, double Mo) {
    double w = 6.65e-29 * N * std::sqrt(2.0 * Ttr / M);
    if (No > 0.0) w += 2.925e-29 * No * std::sqrt(2.0 * Ttr / Mo);
    return w * lam0 * lam0;
}
// Sec. 2.2.1: Voigt HWHM.
double orc_voigt_hwhm(double lamL, double lamG) {
    const double d = (lamL - lamG) / (lamL + lamG);
    return (1.0 - 0.18121 * (1.0 - d * d)
            - (0.023665 * std::exp(0.6 * d) + 0.00418 * std::exp(-1.9 * d)) * std::sin(M_PI * d))
           * (lamL + lamG);
}
// Sec. 2.2.1: Whiting's line shape, um^-1; dlam = |lam - lam0| in nm.
double orc_whiting_phi(double dlam, double lamL, double lamV) {
    const double r = lamL / lamV;
    const double u = dlam / (2.0 * lamV);
    const double u225 = std::pow(u, 2.25);
    const double pre = 1e3 / (2.0 * lamV * (1.065 + 0.447 * r + 0.058 * r * r));
    return pre * ((1.0 - r) * std::exp(-2.772 * u * u)
                  + r / (1.0 + 4.0 * u * u)
                  + 0.016 * r * (1.0 - r) * (std::exp(-0.4 * u225) - 1.0 / (1.0 + 0.1 * u225)));
}

// Strengths and widths of one line in one cell.
//   Sec. 2.2.1 (atoms) / 2.2.2 (molecules): j0 = (hc/4pi) N_u A / (lam 1e-7), times 1e-7 for W.
//   Sec. 2.2.1: kappa0 = j0 / B with B in population form at the line centre (Sec. 2.2).
typedef struct { double Sj, Sk, lamG, lamL, lamV; } orc_line_state;

// Ground-level weight of an atomic species: the summed g of its levels at E = 0.
static double ground_weight(const orc_species* sp, int s) {
    double g = 0.0;
    for (int64_t k = sp->atom_off[s]; k < sp->atom_off[s + 1]; ++k)
        if (sp->atom_E[k] == 0.0) g += sp->atom_g[k];
    return g;
}

static void line_widths(const orc_species* sp, const orc_lines* ln, const orc_cells* cells, const double* lnpref,
                        int64_t l, int64_t c, orc_line_state* st) {
    const int s = ln->species[l];
    const double ne = cells->n[c * cells->ncol + cells->ne_col];
    const bool atom = sp->kind[s] == 0;
    st->lamG = orc_doppler_hwhm(ln->lam0[l], cells->Ttr[c], sp->mass[s]);
    const double lamS0 = (BROAD_FLAGS & 1) && atom ? orc_stark_coeff_ionize(ln->lam0[l], ln->Eu_el[l], BROAD_EION[s])
                                                  : ln->lamS0[l];
    double lamL = orc_lorentz_hwhm(orc_stark_hwhm(lamS0, cells->Tve[c], ne));
    if ((BROAD_FLAGS & 2) && atom && ln->El_el[l] == 0.0 && ln->El_v[l] == 0.0 && ln->El_j[l] == 0.0) {
        const double g0 = ground_weight(sp, s);
        const double N0 = g0 > 0.0 ? std::exp(lnpref[c * sp->S + s] + std::log(g0)) : 0.0;
        lamL += orc_resonance_hwhm(ln->lam0[l], ln->A[l], ln->gu[l], ln->gl[l], N0);
    }
    if ((BROAD_FLAGS & 4) && atom) {
        const int col = sp->dens_col[s];
        const double N = cells->n[c * cells->ncol + col];
        double No = 0.0, NoM = 0.0;
        for (int k = 0; k < cells->ncol && k < BROAD_NCOL; ++k) {
            if (k == col || !(BROAD_COLMASS[k] > 0.0)) continue;
            No += cells->n[c * cells->ncol + k];
            NoM += cells->n[c * cells->ncol + k] * BROAD_COLMASS[k];
        }
        lamL += orc_vdw_hwhm(ln->lam0[l], cells->Ttr[c], N, sp->mass[s], No, No > 0.0 ? NoM / No : 1.0);
    }
    st->lamL = lamL;
    st->lamV = orc_voigt_hwhm(st->lamL, st->lamG);
}

// Sec. 2.1 non-Boltzmann populations (off by default): departure coefficients
// b = N / N_Boltzmann of the collisional-radiative levels, ln b per
// [cell][species][level]; a line whose upper (lower) level has a level index
// >= 0 takes N_u b_u (N_l b_l).
static int64_t DEP_NLEV = 0;
static const double* DEP_LNB = nullptr;
static const int32_t* DEP_LEV_U = nullptr;
static const int32_t* DEP_LEV_L = nullptr;
void orc_set_departures(int64_t n_lev, const double* ln_b, const int32_t* lev_u, const int32_t* lev_l) {
    DEP_NLEV = n_lev; DEP_LNB = ln_b; DEP_LEV_U = lev_u; DEP_LEV_L = lev_l;
}
static double departure(const orc_species* sp, int64_t c, int s, const int32_t* lev, int64_t l) {
    if (!DEP_LNB || !lev || lev[l] < 0) return 0.0;
    return DEP_LNB[(c * sp->S + s) * DEP_NLEV + lev[l]];
}

static void line_strengths(const orc_species* sp, const orc_lines* ln, const orc_cells* cells,
                           const double* lnpref, int64_t l, int64_t c, orc_line_state* st) {
    const int s = ln->species[l];
    const double Ttr = cells->Ttr[c], Tve = cells->Tve[c];
    const double lp = lnpref[c * sp->S + s];
    const double lnNu = orc_ln_level_pop(lp, ln->gu[l], ln->Eu_el[l], ln->Eu_v[l], ln->Eu_j[l], Tve, Ttr) +
                        departure(sp, c, s, DEP_LEV_U, l);
    const double lnNl = orc_ln_level_pop(lp, ln->gl[l], ln->El_el[l], ln->El_v[l], ln->El_j[l], Tve, Ttr) +
                        departure(sp, c, s, DEP_LEV_L, l);
    const double Nu = std::exp(lnNu);
    const double lcm = ln->lam0[l] * 1e-7;
    st->Sj = 1e-7 * (hP * cL / (4.0 * M_PI)) * Nu * ln->A[l] / lcm;
    if (st->Sj == 0.0) {
        st->Sk = 0.0;
    } else {
        // N_l g_u / (N_u g_l) - 1, formed without cancellation
        const double ratio_m1 = std::expm1(lnNl + std::log(ln->gu[l]) - std::log(ln->gl[l]) - lnNu);
        const double B = 1e-7 * 2.0 * hP * cL * cL / (1e4 * std::pow(lcm, 5) * ratio_m1);
        st->Sk = st->Sj / B;
    }
}

static orc_line_state line_state(const orc_species* sp, const orc_lines* ln, const orc_cells* cells,
                                 const double* lnpref, int64_t l, int64_t c) {
    orc_line_state st;
    line_widths(sp, ln, cells, lnpref, l, c, &st);
    line_strengths(sp, ln, cells, lnpref, l, c, &st);
    return st;
}

void orc_line_states(const orc_species* sp, const orc_lines* ln, const orc_cells* cells,
                     const double* lnpref, int64_t c, double* Sj, double* Sk, double* lamG,
                     double* lamL, double* lamV) {
    for (int64_t l = 0; l < ln->L; ++l) {
        orc_line_state st = line_state(sp, ln, cells, lnpref, l, c);
        Sj[l] = st.Sj; Sk[l] = st.Sk; lamG[l] = st.lamG; lamL[l] = st.lamL; lamV[l] = st.lamV;
    }
}

// Grid wavelength lam_k = lam_min + k h, h = (lam_max - lam_min)/(n - 1).
static inline double grid_h(const orc_grid* g) { return (g->lam_max - g->lam_min) / (double)(g->n - 1); }
static inline double grid_lam(const orc_grid* g, int64_t k) { return g->lam_min + (double)k * grid_h(g); }
double orc_grid_lambda(const orc_grid* g, int64_t k) { return grid_lam(g, k); }

// Window: a line contributes to grid point k iff |lam_k - lam0| <= 100 lamV.
static const double WINDOW_HWHM = 100.0;
int orc_in_window(double lam_k, double lam0, double lamV) {
    return std::fabs(lam_k - lam0) <= WINDOW_HWHM * lamV;
}

static inline void neumaier(double& s, double& comp, double x) {
    const double t = s + x;
    if (std::fabs(s) >= std::fabs(x)) comp += (s - t) + x;
    else comp += (x - t) + s;
    s = t;
}

// Number of in-window (line, cell, grid point) triples the last
// orc_spectral_coeffs call evaluated the profile at (a count of work, not a
// step of the method).
static int64_t LAST_EVALUATIONS = 0;
int64_t orc_last_evaluations(void) { return LAST_EVALUATIONS; }

// Line-by-line sums over the grid points [k0, k0 + nk) for every cell:
//   j_k = sum_lines j0 phi(|lam_k - lam0|), kappa_k = sum_lines kappa0 phi(...),
// in-window lines only, lines visited in list order.  Outputs [C][nk].
// kabs (optional) receives sum |kappa0 phi|, the scale of kappa's rounding.
void orc_spectral_coeffs(const orc_species* sp, const orc_lines* ln, const orc_cells* cells,
                         const double* lnpref, const orc_grid* g, int64_t k0, int64_t nk,
                         double* kappa, double* emis, double* kabs) {
    const double h = grid_h(g);
    int64_t evaluations = 0;
#pragma omp parallel reduction(+ : evaluations)
    {
        std::vector<double> sk(nk), ck(nk), sj(nk), cj(nk), sa(nk);
#pragma omp for schedule(dynamic, 1)
        for (int64_t c = 0; c < cells->C; ++c) {
            std::fill(sk.begin(), sk.end(), 0.0); std::fill(ck.begin(), ck.end(), 0.0);
            std::fill(sj.begin(), sj.end(), 0.0); std::fill(cj.begin(), cj.end(), 0.0);
            std::fill(sa.begin(), sa.end(), 0.0);
            for (int64_t l = 0; l < ln->L; ++l) {
                const orc_line_state st = line_state(sp, ln, cells, lnpref, l, c);
                const double lam0 = ln->lam0[l];
                const double half = WINDOW_HWHM * st.lamV;
                // candidate index range, then the literal window test per point
                int64_t a = (int64_t)std::floor((lam0 - half - g->lam_min) / h) - 2;
                int64_t b = (int64_t)std::ceil((lam0 + half - g->lam_min) / h) + 2;
                a = std::max(a, k0);
                b = std::min(b, k0 + nk - 1);
                for (int64_t k = a; k <= b; ++k) {
                    const double lk = grid_lam(g, k);
                    if (!orc_in_window(lk, lam0, st.lamV)) continue;
                    ++evaluations;
                    const double phi = orc_whiting_phi(std::fabs(lk - lam0), st.lamL, st.lamV);
                    neumaier(sj[k - k0], cj[k - k0], st.Sj * phi);
                    neumaier(sk[k - k0], ck[k - k0], st.Sk * phi);
                    sa[k - k0] += std::fabs(st.Sk * phi);
                }
            }
            for (int64_t k = 0; k < nk; ++k) {
                emis[c * nk + k] = sj[k] + cj[k];
                kappa[c * nk + k] = sk[k] + ck[k];
                if (kabs) kabs[c * nk + k] = sa[k];
            }
        }
    }
    LAST_EVALUATIONS = evaluations;
}

// The same sums at individual (cell, k) points, each over the whole line list.
void orc_coeffs_at(const orc_species* sp, const orc_lines* ln, const orc_cells* cells,
                   const double* lnpref, const orc_grid* g, int64_t npts, const int64_t* pc,
                   const int64_t* pk, double* kappa, double* emis, double* kabs) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < npts; ++p) {
        const int64_t c = pc[p], k = pk[p];
        const double lk = grid_lam(g, k);
        double sj = 0, cj = 0, sk = 0, ck = 0, sa = 0;
        for (int64_t l = 0; l < ln->L; ++l) {
            orc_line_state st;
            line_widths(sp, ln, cells, lnpref, l, c, &st);
            if (!orc_in_window(lk, ln->lam0[l], st.lamV)) continue;
            line_strengths(sp, ln, cells, lnpref, l, c, &st);
            const double phi = orc_whiting_phi(std::fabs(lk - ln->lam0[l]), st.lamL, st.lamV);
            neumaier(sj, cj, st.Sj * phi);
            neumaier(sk, ck, st.Sk * phi);
            sa += std::fabs(st.Sk * phi);
        }
        emis[p] = sj + cj;
        kappa[p] = sk + ck;
        if (kabs) kabs[p] = sa;
    }
}

// ---------------------------------------------------------------- geometry ----

// Ray from the surface point (x0, r_body) of a cylinder, direction
// (dx axial, dn outward normal, dt tangential); position at distance t is
// (x0 + t dx, r_body + t dn, t dt), radius sqrt((r_body + t dn)^2 + (t dt)^2).
// Collects every crossing of an x face and an r face, sorts them, and gives
// each segment the cell that holds its midpoint.  Segments are returned from
// the far boundary to the surface point (marching order).  Returns the count
// (or -needed if max_seg is too small).
int64_t orc_axisym_segments(const double* xf, int32_t nx, const double* rf, int32_t nr,
                            double x0, double r_body, double dx, double dn, double dt,
                            int64_t max_seg, int64_t* cell, double* ds) {
    auto radius = [&](double t) { const double y = r_body + t * dn, z = t * dt; return std::sqrt(y * y + z * z); };
    // exit distance: leaving [xf[0], xf[nx]] or reaching rf[nr]
    double t_exit = INFINITY;
    if (dx > 0) t_exit = std::min(t_exit, (xf[nx] - x0) / dx);
    if (dx < 0) t_exit = std::min(t_exit, (xf[0] - x0) / dx);
    const double a = dn * dn + dt * dt, b = 2.0 * r_body * dn;
    auto r_cross = [&](double rr) {   // smallest t >= 0 with radius(t) = rr (rr >= r_body)
        const double cc = r_body * r_body - rr * rr;
        return (-b + std::sqrt(b * b - 4.0 * a * cc)) / (2.0 * a);
    };
    if (a > 0) t_exit = std::min(t_exit, r_cross(rf[nr]));
    std::vector<double> ts;
    ts.push_back(0.0);
    for (int i = 0; i <= nx; ++i) {
        if (dx == 0) break;
        const double t = (xf[i] - x0) / dx;
        if (t > 0 && t < t_exit) ts.push_back(t);
    }
    for (int j = 1; j < nr; ++j) {
        if (a == 0) break;
        const double t = r_cross(rf[j]);
        if (t > 0 && t < t_exit) ts.push_back(t);
    }
    ts.push_back(t_exit);
    std::sort(ts.begin(), ts.end());
    std::vector<std::pair<int64_t, double>> segs;
    for (size_t i = 0; i + 1 < ts.size(); ++i) {
        const double len = ts[i + 1] - ts[i];
        if (!(len > 0)) continue;
        const double tm = 0.5 * (ts[i] + ts[i + 1]);
        const double xm = x0 + tm * dx, rm = radius(tm);
        int64_t ix = std::upper_bound(xf, xf + nx + 1, xm) - xf - 1;
        int64_t jr = std::upper_bound(rf, rf + nr + 1, rm) - rf - 1;
        ix = std::min<int64_t>(std::max<int64_t>(ix, 0), nx - 1);
        jr = std::min<int64_t>(std::max<int64_t>(jr, 0), nr - 1);
        segs.push_back({ix * nr + jr, len});
    }
    const int64_t m = (int64_t)segs.size();
    if (m > max_seg) return -m;
    for (int64_t i = 0; i < m; ++i) {   // reverse: far boundary first
        cell[i] = segs[m - 1 - i].first;
        ds[i] = segs[m - 1 - i].second;
    }
    return m;
}

// ------------------------------------------------------------------- march ----

// Sec. 2.2.3 segment scheme.  A ray crosses cells c_0 (far) ... c_{m-1} (near)
// with lengths ds_i; its nodes sit on the faces: node 0 (far boundary) and node m
// (target point) take the adjacent cell's value, interior node i the mean of
// cells c_{i-1} and c_i.  Over segment i (node i -> node i+1) kappa is held at the
// far node and j is linear, so
//   I_{i+1} = I_i e^{-dtau} + a j_i + b j_{i+1},  dtau = kappa_i ds,
//   a = (f - e^{-dtau}) / kappa_i,  b = (1 - f) / kappa_i,  f = (1 - e^{-dtau}) / dtau,
// the coefficients the paper's integral of the linear emission yields.  For
// |dtau| < thin the coefficients are their series to third order:
//   a = ds (1/2 - dtau/3 + dtau^2/8),  b = ds (1/2 - dtau/6 + dtau^2/24).
// Start: 0 at a far-field boundary, Planck B(T_wall) at a wall (Sec. 2.2.3).
// kappa / emis are [*, ld] tables, columns [0, nk) of the current spectral range;
// `scale` multiplies every ds (1/mu for a slab direction).
// Segment coefficients (far-node coefficient a, near-node coefficient b).
void orc_segment_coeffs(double kap, double s, double thin, double* a, double* b) {
    const double dtau = kap * s;
    if (std::fabs(dtau) < thin) {
        *a = s * (0.5 - dtau / 3.0 + dtau * dtau / 8.0);
        *b = s * (0.5 - dtau / 6.0 + dtau * dtau / 24.0);
    } else {
        const double e = std::exp(-dtau);
        const double f = -std::expm1(-dtau) / dtau;
        *a = (f - e) / kap;
        *b = (1.0 - f) / kap;
    }
}

void orc_march(int64_t m, const int64_t* cell, const double* ds, double scale,
               const double* kappa, const double* emis, int64_t ld, int64_t nk,
               int32_t wall_start, double T_wall, const orc_grid* g, int64_t k0,
               double thin, double* I_out) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nk; ++k) {
        auto node = [&](const double* tab, int64_t i) {
            if (i == 0) return tab[cell[0] * ld + k];
            if (i == m) return tab[cell[m - 1] * ld + k];
            return 0.5 * (tab[cell[i - 1] * ld + k] + tab[cell[i] * ld + k]);
        };
        double I = wall_start ? orc_planck(grid_lam(g, k0 + k), T_wall) : 0.0;
        for (int64_t i = 0; i < m; ++i) {
            const double kap = node(kappa, i);
            const double jf = node(emis, i), jn = node(emis, i + 1);
            const double s = ds[i] * scale;
            double a, b;
            orc_segment_coeffs(kap, s, thin, &a, &b);
            I = I * std::exp(-kap * s) + a * jf + b * jn;
        }
        I_out[k] = I;
    }
}

// Sec. 2.2.3 march on LOS nodes: the tables hold kappa and j at the nodes
// themselves (flow variables interpolated to the node, then the spectral
// coefficients evaluated there).  Segment i runs from node[i] (far) to
// node[i + 1] (near): kappa constant at the far node's value, j linear
// between the two nodes, with the far/near coefficients of orc_segment_coeffs.
void orc_march_nodes(int64_t m, const int64_t* node, const double* ds, const double* kappa, const double* emis,
                     int64_t ld, int64_t nk, int32_t wall_start, double T_wall, const orc_grid* g, int64_t k0,
                     double thin, double* I_out) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nk; ++k) {
        double I = wall_start ? orc_planck(grid_lam(g, k0 + k), T_wall) : 0.0;
        for (int64_t i = 0; i < m; ++i) {
            const double kap = kappa[node[i] * ld + k];
            const double jf = emis[node[i] * ld + k], jn = emis[node[i + 1] * ld + k];
            double a, b;
            orc_segment_coeffs(kap, ds[i], thin, &a, &b);
            I = I * std::exp(-kap * ds[i]) + a * jf + b * jn;
        }
        I_out[k] = I;
    }
}

// Sec. 2.2.3 wall flux, spectral part: trapezoid rule on the uniform grid with
// lam in um (1e-3 per nm); end weights are those of the whole grid, so chunks
// of one grid add up to the full integral.
double orc_spectral_integral(const double* q_lambda, const orc_grid* g, int64_t k0, int64_t nk) {
    const double h_um = grid_h(g) * 1e-3;
    double s = 0.0, comp = 0.0;
    for (int64_t k = 0; k < nk; ++k) {
        const int64_t kk = k0 + k;
        const double w = (kk == 0 || kk == g->n - 1) ? 0.5 : 1.0;
        neumaier(s, comp, w * q_lambda[k] * h_um);
    }
    return s + comp;
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

}  // extern "C"

/*
 * vpmc_oracle.c -- plain, slow, FP64 CPU oracle of the aperture-aware proton
 * Monte Carlo hot path (Feng et al., "Modelling small block aperture in an
 * in-house developed GPU-accelerated Monte Carlo-based dose engine", 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no source,
 * header, table generator or constant with the CUDA path under
 * paper_2307_01416_gb300/csrc; both are written from the same statement of
 * the method (paper Sec. 2.A-2.E plus the physics readings listed in the
 * header comments below).
 *
 * What the method computes, in the paper's order:
 *   Sec. 2.A  every history is created up front with one identical model
 *             (virtual particles: no secondary spawning);
 *   Sec. 2.B  histories cross an optional range shifter (homogeneous slab),
 *             then a 30 mm brass aperture: inside the aperture slab the
 *             crossing-number test decides at every step whether the particle
 *             is in the opening (straight flight, unchanged velocity and
 *             direction) or in brass (state updated from brass physics);
 *   Sec. 2.C  energy is scored into a dose grid or into per-spot
 *             influence-matrix columns;
 *   Sec. 2.E  13 robust scenarios perturb the stopping-power ratio and the
 *             isocentre.
 * The physics of a condensed-history step (Bethe-Bloch tables, Highland
 * scattering, Bohr straggling, 1.2 %/cm nuclear removal, 1 mm / 1 %-energy
 * step rule) is the reading of the engine's physics that this project uses;
 * each reading is stated at the function that implements it.
 *
 * Functions without an independent pin say so in their comment
 * ("parity unpinned").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Physical constants (PDG).                                           */
/* ------------------------------------------------------------------ */
#define ORC_K_BETHE 0.307075     /* 4 pi N_A r_e^2 m_e c^2, MeV cm^2/mol */
#define ORC_ME 0.51099895        /* electron rest energy, MeV            */
#define ORC_MP 938.272           /* proton rest energy, MeV              */
#define ORC_ECUT 0.5             /* transport cut-off, MeV               */
#define ORC_MEV_PER_G_TO_GY 1.602176634e-10
#define ORC_NE 2501              /* energy grid E_k = 0.1 k, k=0..2500   */
#define ORC_NR 4096              /* uniform residual-range grid          */

enum { ORC_WATER = 0, ORC_PMMA = 1, ORC_BRASS = 2, ORC_NMAT = 3 };

/* Material data: Z/A, mean excitation energy (MeV), density (g/cc),
 * radiation length (g/cm^2). */
typedef struct { double za, I, rho, X0; } orc_material;
static const orc_material ORC_MAT[ORC_NMAT] = {
    {0.555087, 75.0e-6, 1.00, 36.08},   /* water                         */
    {0.539369, 74.0e-6, 1.19, 40.55},   /* PMMA range shifter             */
    {0.4573, 330.0e-6, 8.53, 12.9},     /* brass 63 % Cu / 37 % Zn         */
};

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).                  */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 23-bit uniform in (0,1): ((x >> 9) + 1/2) * 2^-23, exactly representable
 * in both FP32 and FP64. */
double orc_uniform(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* Box-Muller: two independent standard normals from two uniforms. */
void orc_box_muller(double u1, double u2, double z[2])
{
    double r = sqrt(-2.0 * log(u1));
    double phi = 2.0 * M_PI * u2;
    z[0] = r * cos(phi);
    z[1] = r * sin(phi);
}

/* RNG stream of one history: key = (seed low word, spot id ^ seed high word);
 * counter = (history, step, slot, 0). */
typedef struct { uint32_t key[2]; uint32_t hist; } orc_stream;

static void stream_block(const orc_stream* st, uint32_t step, uint32_t slot, double u[4])
{
    uint32_t ctr[4] = {st->hist, step, slot, 0u}, x[4];
    orc_philox4x32_10(ctr, st->key, x);
    for (int i = 0; i < 4; ++i) u[i] = orc_uniform(x[i]);
}

/* Six 21-bit uniforms of one condensed-history step from one Philox block,
 * counter (history, step, 1, 0): the top 21 bits of words 0..3 give u0..u3;
 * the low 11 bits of word 0 (or 2) followed by the low 10 bits of word 1 (or
 * 3) give u4 (or u5).  u = (v + 1/2) 2^-21 lies in (0, 1) and is exact in
 * binary32.  Scattering takes the Box-Muller pairs (u0, u1), (u2, u3);
 * straggling the first normal of (u4, u5). */
void orc_step_uniforms(uint32_t hist, uint32_t step, const uint32_t key[2], double u[6])
{
    uint32_t ctr[4] = {hist, step, 1u, 0u}, x[4];
    orc_philox4x32_10(ctr, key, x);
    const double sc = ldexp(1.0, -21);
    for (int i = 0; i < 4; ++i) u[i] = ((double)(x[i] >> 11) + 0.5) * sc;
    u[4] = ((double)(((x[0] & 0x7FFu) << 10) | (x[1] & 0x3FFu)) + 0.5) * sc;
    u[5] = ((double)(((x[2] & 0x7FFu) << 10) | (x[3] & 0x3FFu)) + 0.5) * sc;
}

/* The same six uniforms at 32-bit resolution, u = (x + 1/2) 2^-32, from two
 * blocks: counter (history, step, 1, 0) words 0..3 give u0..u3, counter
 * (history, step, 2, 0) words 0, 1 give u4, u5.  Box-Muller normals then
 * reach sqrt(-2 ln 2^-33) = 6.8 sigma instead of 5.5 sigma.  Not an engine
 * stream: only the study of the 21-bit lattice uses it. */
static void orc_step_uniforms_fine(uint32_t hist, uint32_t step, const uint32_t key[2], double u[6])
{
    uint32_t c1[4] = {hist, step, 1u, 0u}, c2[4] = {hist, step, 2u, 0u}, x[4], y[4];
    orc_philox4x32_10(c1, key, x);
    orc_philox4x32_10(c2, key, y);
    const double sc = ldexp(1.0, -32);
    for (int i = 0; i < 4; ++i) u[i] = ((double)x[i] + 0.5) * sc;
    u[4] = ((double)y[0] + 0.5) * sc;
    u[5] = ((double)y[1] + 0.5) * sc;
}

/* Four normals from one Philox block (two Box-Muller pairs). */
static void stream_normals4(const orc_stream* st, uint32_t step, uint32_t slot, double z[4])
{
    double u[4];
    stream_block(st, step, slot, u);
    orc_box_muller(u[0], u[1], z);
    orc_box_muller(u[2], u[3], z + 2);
}

/* ------------------------------------------------------------------ */
/* Stopping power and range tables.                                    */
/* ------------------------------------------------------------------ */
/* Bethe-Bloch mass electronic stopping power, MeV cm^2/g, without shell or
 * density-effect corrections, with the full T_max. */
double orc_stopping_power(int mat, double T)
{
    const orc_material* m = &ORC_MAT[mat];
    double gamma = 1.0 + T / ORC_MP;
    double beta2 = 1.0 - 1.0 / (gamma * gamma);
    double bg2 = beta2 * gamma * gamma;
    double ratio = ORC_ME / ORC_MP;
    double tmax = 2.0 * ORC_ME * bg2 / (1.0 + 2.0 * gamma * ratio + ratio * ratio);
    double arg = 2.0 * ORC_ME * bg2 * tmax / (m->I * m->I);
    return ORC_K_BETHE * m->za / beta2 * (0.5 * log(arg) - beta2);
}

typedef struct {
    double R[ORC_NE];     /* R(E_k), mm * g/cc (areal range times 10)       */
    double Einv[ORC_NR];  /* E at R_j = j * dR                              */
    double dR;
} orc_table;

static orc_table g_tab[ORC_NMAT];
static int g_tab_ready = 0;

/* Integrand of the CSDA range in mm*g/cc per MeV. */
static double range_integrand(int mat, double E) { return 10.0 / orc_stopping_power(mat, E); }

/* Composite Simpson over [a, b] with n (even) sub-intervals. */
static double simpson(int mat, double a, double b, int n)
{
    double h = (b - a) / n;
    double s = range_integrand(mat, a) + range_integrand(mat, b);
    for (int i = 1; i < n; ++i) s += (i & 1 ? 4.0 : 2.0) * range_integrand(mat, a + i * h);
    return s * h / 3.0;
}

static void build_table(int mat, orc_table* t)
{
    /* R(E_k) = integral_{E_cut}^{E_k} dE / S(E), 0.001 MeV Simpson sub-grid. */
    t->R[0] = 0.0;
    for (int k = 1; k < ORC_NE; ++k) {
        double lo = 0.1 * (k - 1), hi = 0.1 * k;
        if (hi <= ORC_ECUT) { t->R[k] = 0.0; continue; }
        if (lo < ORC_ECUT) lo = ORC_ECUT;
        t->R[k] = t->R[k - 1] + simpson(mat, lo, hi, 100);
    }
    /* E(R) on a uniform R grid: inverse of the piecewise-linear R(E). */
    double rmax = t->R[ORC_NE - 1];
    t->dR = rmax / (ORC_NR - 1);
    int k = 0;
    for (int j = 0; j < ORC_NR; ++j) {
        double r = j * t->dR;
        if (j == ORC_NR - 1) { t->Einv[j] = 0.1 * (ORC_NE - 1); break; }
        if (r <= 0.0) { t->Einv[j] = ORC_ECUT; continue; }
        while (k + 1 < ORC_NE - 1 && t->R[k + 1] < r) ++k;
        /* now R[k] < r <= R[k+1] (R[k] may be 0 below the cut) */
        double f = (r - t->R[k]) / (t->R[k + 1] - t->R[k]);
        double e0 = 0.1 * k;
        if (e0 < ORC_ECUT) e0 = ORC_ECUT;   /* R is 0 up to the cut */
        t->Einv[j] = e0 + f * (0.1 * (k + 1) - e0);
    }
}

void orc_init_tables(void)
{
    if (g_tab_ready) return;
    for (int m = 0; m < ORC_NMAT; ++m) build_table(m, &g_tab[m]);
    g_tab_ready = 1;
}

double orc_table_R(int mat, int k) { orc_init_tables(); return g_tab[mat].R[k]; }
double orc_table_Einv(int mat, int j) { orc_init_tables(); return g_tab[mat].Einv[j]; }
double orc_table_dR(int mat) { orc_init_tables(); return g_tab[mat].dR; }

/* Residual range R(E) by linear interpolation on the 0.1 MeV grid. */
double orc_range(int mat, double E)
{
    const orc_table* t = &g_tab[mat];
    if (E <= 0.0) return 0.0;
    double x = E * 10.0;
    int i = (int)floor(x);
    if (i > ORC_NE - 2) i = ORC_NE - 2;
    double f = x - i;
    return t->R[i] + f * (t->R[i + 1] - t->R[i]);
}

/* Energy E(R) by linear interpolation on the uniform R grid. */
double orc_energy(int mat, double R)
{
    const orc_table* t = &g_tab[mat];
    if (R <= 0.0) return ORC_ECUT;
    double x = R / t->dR;
    int j = (int)floor(x);
    if (j > ORC_NR - 2) j = ORC_NR - 2;
    double f = x - j;
    return t->Einv[j] + f * (t->Einv[j + 1] - t->Einv[j]);
}

/* Linear stopping-power ratio of PMMA to water at energy T. */
double orc_spr_pmma(double T)
{
    return orc_stopping_power(ORC_PMMA, T) * ORC_MAT[ORC_PMMA].rho / orc_stopping_power(ORC_WATER, T);
}

/* ------------------------------------------------------------------ */
/* HU -> (mass density, stopping-power ratio): 4-segment curve.        */
/* ------------------------------------------------------------------ */
typedef struct { double hu[5], rho[5], spr[5]; } orc_curve;

void orc_hu_props(const orc_curve* c, double hu, double* rho, double* spr)
{
    double h = hu;
    if (h < c->hu[0]) h = c->hu[0];
    if (h > 3071.0) h = 3071.0;
    int s = 0;
    while (s < 3 && h >= c->hu[s + 1]) ++s;
    double f = (h - c->hu[s]) / (c->hu[s + 1] - c->hu[s]);
    *rho = c->rho[s] + f * (c->rho[s + 1] - c->rho[s]);
    *spr = c->spr[s] + f * (c->spr[s + 1] - c->spr[s]);
}

/* ------------------------------------------------------------------ */
/* Aperture geometry: crossing-number test (paper Sec. 2.B, ref [67]). */
/* ------------------------------------------------------------------ */
/* poly: n vertices, xy interleaved, BEV mm.  Half-open edge rule. */
int orc_point_in_polygon(const double* poly, int n, double x, double y)
{
    int inside = 0;
    for (int i = 0, j = n - 1; i < n; j = i++) {
        double xi = poly[2 * i], yi = poly[2 * i + 1];
        double xj = poly[2 * j], yj = poly[2 * j + 1];
        if ((yi > y) != (yj > y)) {
            double xc = xi + (y - yi) * (xj - xi) / (yj - yi);
            if (x < xc) inside = !inside;
        }
    }
    return inside;
}

/* Smallest s > 0 at which (x, y) + s (dx, dy) crosses a polygon edge. */
double orc_first_wall_hit(const double* poly, int n, double x, double y, double dx, double dy)
{
    double best = INFINITY;
    for (int i = 0; i < n; ++i) {
        int j = (i + 1) % n;
        double ex = poly[2 * j] - poly[2 * i], ey = poly[2 * j + 1] - poly[2 * i + 1];
        double den = dx * ey - dy * ex;
        if (den == 0.0) continue;
        double wx = poly[2 * i] - x, wy = poly[2 * i + 1] - y;
        double s = (wx * ey - wy * ex) / den;
        double lam = (wx * dy - wy * dx) / den;
        if (s > 0.0 && lam >= 0.0 && lam <= 1.0 && s < best) best = s;
    }
    return best;
}


/* Distance from (x, y) to the polygon boundary. */
double orc_wall_distance(const double* poly, int n, double x, double y)
{
    double best = INFINITY;
    for (int i = 0; i < n; ++i) {
        int j = (i + 1) % n;
        double ax = poly[2 * i], ay = poly[2 * i + 1];
        double ex = poly[2 * j] - ax, ey = poly[2 * j + 1] - ay;
        double t = ((x - ax) * ex + (y - ay) * ey) / (ex * ex + ey * ey);
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
        double dx = ax + t * ex - x, dy = ay + t * ey - y;
        double d = sqrt(dx * dx + dy * dy);
        if (d < best) best = d;
    }
    return best;
}

/* ------------------------------------------------------------------ */
/* Problem description (the oracle's own structs).                     */
/* ------------------------------------------------------------------ */
typedef struct { int nx, ny, nz; double dx, dy, dz, ox, oy, oz; } orc_grid;

typedef struct {
    double dir[3], bevx[3], iso[3];   /* beam axis w, BEV x axis u, isocentre */
    double source_to_iso;             /* source plane at t = -source_to_iso   */
    int rs_present;
    double rs_wet, rs_radius, rs_down_to_iso;
    int ap_present;
    double ap_thickness, ap_down_to_iso;
    int poly_offset, nvert;           /* vertices in the shared xy array      */
    double ap_sad;                    /* divergent walls: virtual source at
                                         t = -ap_sad (0: walls parallel to
                                         the beam axis)                       */
} orc_beam;

/* ------------------------------------------------------------------ */
/* Divergent aperture walls (the authors' next step, Sec. 4).  Reading:  */
/* the polygon is the opening at the block's downstream face t_dn; each  */
/* wall is the plane through the virtual source S = (0, 0, -sad) and one */
/* polygon edge there, so the opening at depth t is the polygon scaled   */
/* by (t + sad) / (t_dn + sad).  ap_sad = 0 keeps parallel walls.        */
/* ------------------------------------------------------------------ */

/* Scale of the opening at depth t relative to the downstream face. */
static double ap_scale(const orc_beam* bm, double t)
{
    if (!(bm->ap_sad > 0.0)) return 1.0;
    double tdn = -bm->ap_down_to_iso;
    return (t + bm->ap_sad) / (tdn + bm->ap_sad);
}

/* Is (x, y, t) inside the opening? */
static int ap_in_opening(const orc_beam* bm, const double* poly, double x, double y, double t)
{
    double s = ap_scale(bm, t);
    return orc_point_in_polygon(poly, bm->nvert, x / s, y / s);
}

/* Wall distance used by the tie flag and the range rejection: the distance,
 * in the plane of constant depth through the point, to the opening's
 * contour at that depth, times the cosine of the largest wall tilt, so that
 * it never exceeds the 3D distance to a wall (parallel walls: the plain 2D
 * distance). */
static double ap_wall_distance(const orc_beam* bm, const double* poly, double x, double y, double t)
{
    if (!(bm->ap_sad > 0.0)) return orc_wall_distance(poly, bm->nvert, x, y);
    double s = ap_scale(bm, t);
    double K = -bm->ap_down_to_iso + bm->ap_sad, rc = 0.0;
    for (int i = 0; i < bm->nvert; ++i) {
        double r = hypot(poly[2 * i], poly[2 * i + 1]);
        if (r > rc) rc = r;
    }
    return s * orc_wall_distance(poly, bm->nvert, x / s, y / s) * (K / sqrt(K * K + rc * rc));
}

/* Smallest s > 0 at which p + s d meets a wall: each wall is the plane
 * through S and the edge (A, B) at t_dn; the hit must lie between the
 * plane's two edge rays (its projection from S onto t_dn falls on the edge).
 * Parallel walls: the 2D ray-edge test. */
static double ap_first_wall_hit(const orc_beam* bm, const double* poly, const double p[3], const double d[3])
{
    if (!(bm->ap_sad > 0.0)) return orc_first_wall_hit(poly, bm->nvert, p[0], p[1], d[0], d[1]);
    double tdn = -bm->ap_down_to_iso, sad = bm->ap_sad;
    double S[3] = {0.0, 0.0, -sad};
    double best = INFINITY;
    for (int i = 0; i < bm->nvert; ++i) {
        int j = (i + 1) % bm->nvert;
        double A[3] = {poly[2 * i], poly[2 * i + 1], tdn}, B[3] = {poly[2 * j], poly[2 * j + 1], tdn};
        double a[3], b[3], n[3];
        for (int k = 0; k < 3; ++k) { a[k] = A[k] - S[k]; b[k] = B[k] - S[k]; }
        n[0] = a[1] * b[2] - a[2] * b[1];
        n[1] = a[2] * b[0] - a[0] * b[2];
        n[2] = a[0] * b[1] - a[1] * b[0];
        double den = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
        if (den == 0.0) continue;
        double s = (n[0] * (A[0] - p[0]) + n[1] * (A[1] - p[1]) + n[2] * (A[2] - p[2])) / den;
        if (!(s > 0.0) || s >= best) continue;
        double q[3] = {p[0] + s * d[0], p[1] + s * d[1], p[2] + s * d[2]};
        double f = (tdn + sad) / (q[2] + sad);           /* project from S onto t_dn */
        double qx = q[0] * f, qy = q[1] * f;
        double ex = B[0] - A[0], ey = B[1] - A[1];
        double lam = ((qx - A[0]) * ex + (qy - A[1]) * ey) / (ex * ex + ey * ey);
        if (lam >= 0.0 && lam <= 1.0) best = s;
    }
    return best;
}

/* Test hook: (in the opening, first wall hit, wall distance) of a point and
 * direction for a beam's aperture; poly is that beam's polygon. */
void orc_aperture_query(const orc_beam* bm, const double* poly, const double p[3], const double d[3], double out[3])
{
    out[0] = ap_in_opening(bm, poly, p[0], p[1], p[2]);
    out[1] = ap_first_wall_hit(bm, poly, p, d);
    out[2] = ap_wall_distance(bm, poly, p[0], p[1], p[2]);
}

typedef struct {
    int beam;
    int spot_key;           /* spot id in the RNG key                        */
    double energy, x, y, sigma, div_mrad;
    int64_t h_begin, n_hist;
    double weight;
} orc_spot;

typedef struct { double shift[3]; double spr_scale; } orc_scen;

typedef struct {
    uint64_t seed;
    int mcs, straggling, nuclear;
    int frac_bits;
    int fine_uniforms;      /* 1: the step's six uniforms at 32-bit resolution (a study of reading c17's
                               21-bit lattice); 0: the engines' 21-bit lattice */
} orc_opts;

typedef struct {
    const orc_grid* ct;
    const int16_t* hu;
    const orc_curve* curve;
    const orc_grid* sg;     /* scoring grid, same extent as ct */
    const orc_beam* beams;
    const double* poly_xy;
} orc_problem;

enum { FATE_STOP = 0, FATE_NUC = 1, FATE_LEAK = 2, FATE_RS = 3, FATE_AP = 4, FATE_ERR = 5 };

typedef struct {
    int32_t fate;
    int32_t steps;      /* condensed-history steps of the history            */
    double e_dep;       /* energy scored in the patient grid, MeV            */
    double e_end;       /* kinetic energy when it left, MeV                  */
    double pos[3];      /* end position, patient coordinates, mm             */
    int64_t q_dep;      /* sum of the history's fixed-point grid deposits    */
    int32_t flags;      /* bit 0: a step started within ORC_TIE_MM of an
                           aperture wall; bit 1: of the range-shifter rim;
                           bit 2: nuclear removal in a medium below
                           ORC_LOW_RHO g/cc (the interaction point moves by
                           (free-path rounding) / (0.0012 rho) mm);
                           bit 3: a CT voxel face crossed at a direction
                           cosine below 0.01 |delta SPR| (the crossing point
                           moves by (position rounding) / cosine);
                           bit 4: unused;
                           bit 5: the end point is ill-conditioned: moving
                           the start by ORC_COND_MM moves it by more than
                           1e-4 of the track;
                           bit 6: so are the fate or the scored energy      */
    int32_t pad;
    double path;        /* path length travelled in the patient grid, mm     */
    double track;       /* whole track length from the source plane, mm      */
} orc_record;

/* Distance below which a device boundary makes a history ill-conditioned:
 * at grazing incidence a rounding-level shift of the position changes which
 * side of the boundary a step starts on. */
#define ORC_TIE_MM 0.01
#define ORC_LOW_RHO 0.1

/* Tallies: 0 energy in, 1 scored in grid, 2 leaked, 3 range shifter,
 * 4 aperture, 5 nuclear (included in 1, 3, 4), 6 histories, 7 steps,
 * 8 histories stopped by the iteration cap. */
#define ORC_NTALLY 9

/* ------------------------------------------------------------------ */
/* One condensed-history step (range shifter, brass and patient alike). */
/* ------------------------------------------------------------------ */
typedef struct {
    int table;      /* range/energy table                              */
    double kappa;   /* table units (mm*g/cc) consumed per mm of path   */
    double rho;     /* mass density, g/cc                              */
    double za;      /* Z/A for straggling                              */
    double X0;      /* radiation length, g/cm^2                        */
} orc_medium;

typedef struct {
    double p[3], d[3];
    double E, nlam;
    double R;           /* residual range in the current medium's table units */
    uint32_t step;
} orc_particle;

enum { LIM_NONE = 0, LIM_GEOM = 1, LIM_NUC = 2 };

typedef struct {
    double s;           /* step length, mm                      */
    double dE;          /* deposited energy, MeV                */
    int limiter;
    int killed;         /* 1 stopped at the cut-off, 2 nuclear   */
    double disp[3];     /* lateral displacement from scattering  */
} orc_step;

/* Duff et al. 2017, "Building an orthonormal basis, revisited". */
static void orthonormal_basis(const double n[3], double b1[3], double b2[3])
{
    double sign = copysign(1.0, n[2]);
    double a = -1.0 / (sign + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1.0 + sign * n[0] * n[0] * a; b1[1] = sign * b; b1[2] = -sign * n[0];
    b2[0] = b; b2[1] = sign + n[1] * n[1] * a; b2[2] = -n[1];
}

/* Highland width (PDG form) for a step of s mm in medium med at energy T. */
double orc_highland(double T, double s_mm, double rho, double X0)
{
    double x = s_mm * rho / (X0 * 10.0);
    if (x < 1e-6) return 0.0;
    double bcp = T * (T + 2.0 * ORC_MP) / (T + ORC_MP);
    return 13.6 / bcp * sqrt(x) * (1.0 + 0.038 * log(x));
}

/* Bohr straggling variance (MeV^2) for s mm at energy T. */
double orc_bohr_var(double T, double s_mm, double rho, double za)
{
    double gamma = 1.0 + T / ORC_MP;
    double beta2 = 1.0 - 1.0 / (gamma * gamma);
    return 0.1569 * rho * za * (s_mm * 0.1) * (1.0 - 0.5 * beta2) / (1.0 - beta2);
}

static void ch_step(const orc_medium* med, orc_particle* pt, double s_geom,
                    const orc_opts* op, const orc_stream* st, orc_step* out)
{
    double E = pt->E;
    /* step rule: min(1 mm, 1 % energy loss, geometry, nuclear point).  The
     * residual range R0 is carried with the particle inside one medium so
     * that the CSDA range is conserved exactly by the table lookups. */
    double R0 = pt->R;
    double s1 = (R0 - orc_range(med->table, 0.99 * E)) / med->kappa;
    if (!(s1 > 0.0)) s1 = R0 / med->kappa;
    double mu = op->nuclear ? 0.0012 * med->rho : 0.0;
    double s = 1.0;
    int lim = LIM_NONE;
    if (s1 < s) s = s1;
    if (s_geom < s) { s = s_geom; lim = LIM_GEOM; }
    if (mu > 0.0) {
        double snuc = pt->nlam / mu;
        if (snuc < s) { s = snuc; lim = LIM_NUC; }
    }
    pt->step += 1;
    if (lim == LIM_NUC) pt->nlam = 0.0; else pt->nlam -= mu * s;

    /* mean energy loss from the range table (CSDA) */
    double R1 = R0 - s * med->kappa;
    double Emean = R1 > 0.0 ? orc_energy(med->table, R1) : ORC_ECUT;
    double dE = E - Emean;
    double u[6];
    if (op->mcs || op->straggling) {
        if (op->fine_uniforms) orc_step_uniforms_fine(st->hist, pt->step, st->key, u);
        else orc_step_uniforms(st->hist, pt->step, st->key, u);
    }
    if (op->straggling) {
        double z[2];
        orc_box_muller(u[4], u[5], z);
        dE += sqrt(orc_bohr_var(E, s, med->rho, med->za)) * z[0];
    }
    if (dE < 0.0) dE = 0.0;
    if (dE > E) dE = E;
    double Enew = E - dE;
    /* carried range: R1, corrected by the range equivalent of the straggling */
    double Rnew = R1;
    if (op->straggling) {
        Rnew = R1 + (orc_range(med->table, Enew) - orc_range(med->table, Emean));
        if (!(Rnew > 0.0)) Rnew = orc_range(med->table, Enew);
    }
    pt->R = Rnew;

    out->s = s;
    out->limiter = lim;
    out->disp[0] = out->disp[1] = out->disp[2] = 0.0;
    out->killed = 0;
    if (lim == LIM_NUC) out->killed = 2;
    else if (Enew <= ORC_ECUT) out->killed = 1;
    if (out->killed) { out->dE = E; pt->E = 0.0; }
    else { out->dE = dE; pt->E = Enew; }

    /* advance along the direction at the start of the step */
    for (int k = 0; k < 3; ++k) pt->p[k] += s * pt->d[k];

    if (op->mcs && !out->killed) {
        double theta0 = orc_highland(E, s, med->rho, med->X0);
        double z[4];
        orc_box_muller(u[0], u[1], z);
        orc_box_muller(u[2], u[3], z + 2);
        /* two projected planes, each a correlated (angle, offset) pair */
        double th1 = z[1] * theta0, th2 = z[3] * theta0;
        double dx1 = s * theta0 * (z[0] / sqrt(12.0) + 0.5 * z[1]);
        double dx2 = s * theta0 * (z[2] / sqrt(12.0) + 0.5 * z[3]);
        double e1[3], e2[3];
        orthonormal_basis(pt->d, e1, e2);
        for (int k = 0; k < 3; ++k) out->disp[k] = dx1 * e1[k] + dx2 * e2[k];
        double th = sqrt(th1 * th1 + th2 * th2);
        double c = cos(th), sc = th > 0.0 ? sin(th) / th : 1.0;
        double nd[3], nn = 0.0;
        for (int k = 0; k < 3; ++k) { nd[k] = c * pt->d[k] + sc * (th1 * e1[k] + th2 * e2[k]); nn += nd[k] * nd[k]; }
        nn = sqrt(nn);
        for (int k = 0; k < 3; ++k) pt->d[k] = nd[k] / nn;
    }
}

/* ------------------------------------------------------------------ */
/* One history (paper Sec. 2.A, 2.B, 2.E).                             */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_problem* pb;
    const orc_scen* sc;
    const orc_opts* op;
    int mode;               /* 0 dose grid (weighted), 1 per-spot columns */
    int64_t* q;             /* deposit target (NULL: score nothing)       */
    int64_t nvox;
} orc_run_ctx;

#define ORC_MAX_ITER 200000

static void beam_axes(const orc_beam* bm, double u[3], double v[3], double w[3])
{
    for (int k = 0; k < 3; ++k) { w[k] = bm->dir[k]; u[k] = bm->bevx[k]; }
    v[0] = w[1] * u[2] - w[2] * u[1];
    v[1] = w[2] * u[0] - w[0] * u[2];
    v[2] = w[0] * u[1] - w[1] * u[0];
}

static void bev_to_patient(const orc_beam* bm, const orc_scen* sc, const double pb[3], double out[3])
{
    double u[3], v[3], w[3];
    beam_axes(bm, u, v, w);
    for (int k = 0; k < 3; ++k) out[k] = bm->iso[k] + sc->shift[k] + pb[0] * u[k] + pb[1] * v[k] + pb[2] * w[k];
}

/* Aperture block (paper Sec. 2.B) from the particle's state upstream of
 * it: a straight drift to the entrance plane, then at every step the
 * crossing-number test.  In the opening the particle keeps its velocity and
 * direction up to a wall or the exit plane; a wall hit forces the next step
 * into brass.  In brass it takes a condensed-history step with brass
 * physics.  Returns 0 when it leaves through the exit plane, else FATE_AP
 * (absorbed: stopped or nuclear removal), FATE_LEAK (left
 * upstream) or FATE_ERR (iteration cap). */
static int aperture_block(const orc_beam* bm, const double* poly, orc_particle* pt, const orc_opts* op,
                          orc_stream* st, orc_record* rec, double* tl, long* iter)
{
    double tdn = -bm->ap_down_to_iso, tup = tdn - bm->ap_thickness;
    if (pt->d[2] <= 0.0) return FATE_LEAK;
    double sdr = (tup - pt->p[2]) / pt->d[2];
    for (int k = 0; k < 3; ++k) pt->p[k] += sdr * pt->d[k];
    rec->track += sdr;
    orc_medium med = {ORC_BRASS, ORC_MAT[ORC_BRASS].rho, ORC_MAT[ORC_BRASS].rho, ORC_MAT[ORC_BRASS].za, ORC_MAT[ORC_BRASS].X0};
    orc_step so;
    int forced_brass = 0;
    pt->R = orc_range(ORC_BRASS, pt->E);
    for (;;) {
        if (++*iter > ORC_MAX_ITER) return FATE_ERR;
        double sg = INFINITY;
        int down = 1;
        if (pt->d[2] > 0.0) sg = (tdn - pt->p[2]) / pt->d[2];
        else if (pt->d[2] < 0.0) { sg = (tup - pt->p[2]) / pt->d[2]; down = 0; }
        if (sg < 0.0) sg = 0.0;   /* scattering offsets can leave it past the plane */
        if (ap_wall_distance(bm, poly, pt->p[0], pt->p[1], pt->p[2]) < ORC_TIE_MM) rec->flags |= 1;
        int in_open = !forced_brass && ap_in_opening(bm, poly, pt->p[0], pt->p[1], pt->p[2]);
        if (in_open) {
            /* opening: keep velocity and direction up to a wall or the exit */
            double sw = ap_first_wall_hit(bm, poly, pt->p, pt->d);
            if (sw < sg) {
                for (int k = 0; k < 3; ++k) pt->p[k] += sw * pt->d[k];
                rec->track += sw;
                forced_brass = 1;
                continue;
            }
            if (!isfinite(sg)) return FATE_ERR;
            for (int k = 0; k < 3; ++k) pt->p[k] += sg * pt->d[k];
            rec->track += sg;
            return down ? 0 : FATE_LEAK;
        }
        /* brass: condensed-history step with brass physics */
        forced_brass = 0;
        ch_step(&med, pt, sg, op, st, &so);
        rec->track += so.s;
        tl[4] += so.dE;
        tl[7] += 1.0;
        rec->steps += 1;
        if (so.killed) {
            if (so.killed == 2) tl[5] += so.dE;
            return FATE_AP;
        }
        for (int k = 0; k < 3; ++k) pt->p[k] += so.disp[k];
        if (so.limiter == LIM_GEOM) return down ? 0 : FATE_LEAK;
    }
}

static void transport_history(orc_run_ctx* rc, const orc_spot* sp, int spot_index, int64_t h,
                              orc_record* rec, double* tl, const double* shift)
{
    const orc_problem* pb = rc->pb;
    const orc_beam* bm = &pb->beams[sp->beam];
    const orc_opts* op = rc->op;
    const double fscale = ldexp(1.0, op->frac_bits);
    orc_stream st;
    st.key[0] = (uint32_t)op->seed;
    st.key[1] = (uint32_t)(op->seed >> 32) ^ (uint32_t)sp->spot_key;
    st.hist = (uint32_t)h;

    orc_particle pt;
    memset(&pt, 0, sizeof pt);
    memset(rec, 0, sizeof *rec);
    rec->fate = FATE_ERR;

    /* source (slot 0, step 0): (x, y) at the isocentre plane and two
     * projected angles; slot 3 gives the nuclear mean-free-path count. */
    double z[4];
    stream_normals4(&st, 0u, 0u, z);
    double a0 = sp->x + sp->sigma * z[0];
    double b0 = sp->y + sp->sigma * z[1];
    if (shift) { a0 += shift[0]; b0 += shift[1]; }
    double tha = sp->div_mrad * 1e-3 * z[2];
    double thb = sp->div_mrad * 1e-3 * z[3];
    double nrm = sqrt(1.0 + tha * tha + thb * thb);
    double tsrc = -bm->source_to_iso;
    /* BEV coordinates (a, b, t): t along the beam, origin at isocentre */
    pt.d[0] = tha / nrm; pt.d[1] = thb / nrm; pt.d[2] = 1.0 / nrm;
    pt.p[0] = a0 + tsrc * tha; pt.p[1] = b0 + tsrc * thb; pt.p[2] = tsrc;
    pt.E = sp->energy;
    if (op->nuclear) {
        double u[4];
        stream_block(&st, 0u, 3u, u);
        pt.nlam = -log(u[0]);
    } else {
        pt.nlam = INFINITY;
    }
    tl[0] += pt.E;
    tl[6] += 1.0;

    long iter = 0;
    int in_patient = 0;
    double P[3] = {0, 0, 0};
    orc_step so;

    /* ---- range shifter: homogeneous slab of finite radius ---- */
    if (bm->rs_present) {
        double thick = bm->rs_wet / orc_spr_pmma(150.0);
        double tdn = -bm->rs_down_to_iso, tup = tdn - thick;
        double sdr = (tup - pt.p[2]) / pt.d[2];
        for (int k = 0; k < 3; ++k) pt.p[k] += sdr * pt.d[k];
        rec->track += sdr;
        orc_medium med = {ORC_PMMA, ORC_MAT[ORC_PMMA].rho, ORC_MAT[ORC_PMMA].rho, ORC_MAT[ORC_PMMA].za, ORC_MAT[ORC_PMMA].X0};
        pt.R = orc_range(ORC_PMMA, pt.E);
        for (;;) {
            if (++iter > ORC_MAX_ITER) goto fail;
            double r2 = pt.p[0] * pt.p[0] + pt.p[1] * pt.p[1];
            if (fabs(sqrt(r2) - bm->rs_radius) < ORC_TIE_MM) rec->flags |= 2;
            if (r2 > bm->rs_radius * bm->rs_radius) {
                /* outside the shifter: straight flight to its exit plane */
                if (pt.d[2] <= 0.0) goto leak;
                double sf = (tdn - pt.p[2]) / pt.d[2];
                for (int k = 0; k < 3; ++k) pt.p[k] += sf * pt.d[k];
                rec->track += sf;
                break;
            }
            double sg = INFINITY;
            int down = 1;
            if (pt.d[2] > 0.0) sg = (tdn - pt.p[2]) / pt.d[2];
            else if (pt.d[2] < 0.0) { sg = (tup - pt.p[2]) / pt.d[2]; down = 0; }
            if (sg < 0.0) sg = 0.0;   /* scattering offsets can leave it past the plane */
            ch_step(&med, &pt, sg, op, &st, &so);
            rec->track += so.s;
            tl[3] += so.dE;
            tl[7] += 1.0;
            rec->steps += 1;
            if (so.killed) {
                if (so.killed == 2) tl[5] += so.dE;
                rec->fate = FATE_RS;
                goto done;
            }
            for (int k = 0; k < 3; ++k) pt.p[k] += so.disp[k];
            if (so.limiter == LIM_GEOM) {
                if (!down) goto leak;
                break;
            }
        }
    }

    /* ---- aperture block (paper Sec. 2.B) ---- */
    if (bm->ap_present) {
        int r = aperture_block(bm, pb->poly_xy + 2 * (int64_t)bm->poly_offset, &pt, op, &st, rec, tl, &iter);
        if (r == FATE_LEAK) goto leak;
        if (r == FATE_ERR) goto fail;
        if (r == FATE_AP) { rec->fate = FATE_AP; goto done; }
    }

    /* ---- patient / phantom grid ---- */
    {
        const orc_grid* g = pb->ct;
        const orc_grid* sgd = pb->sg;
        double u[3], v[3], w[3], D[3];
        beam_axes(bm, u, v, w);
        for (int k = 0; k < 3; ++k) {
            P[k] = bm->iso[k] + rc->sc->shift[k] + pt.p[0] * u[k] + pt.p[1] * v[k] + pt.p[2] * w[k];
            D[k] = pt.d[0] * u[k] + pt.d[1] * v[k] + pt.d[2] * w[k];
        }
        in_patient = 1;
        const double lo[3] = {g->ox, g->oy, g->oz};
        const int n[3] = {g->nx, g->ny, g->nz};
        const double dl[3] = {g->dx, g->dy, g->dz};
        const int ns[3] = {sgd->nx, sgd->ny, sgd->nz};
        const double dls[3] = {sgd->dx, sgd->dy, sgd->dz};
        double hi[3];
        for (int k = 0; k < 3; ++k) hi[k] = lo[k] + n[k] * dl[k];
        /* ray / box entry */
        double tmin = -INFINITY, tmax = INFINITY;
        for (int k = 0; k < 3; ++k) {
            if (D[k] != 0.0) {
                double t1 = (lo[k] - P[k]) / D[k], t2 = (hi[k] - P[k]) / D[k];
                if (t1 > t2) { double tt = t1; t1 = t2; t2 = tt; }
                if (t1 > tmin) tmin = t1;
                if (t2 < tmax) tmax = t2;
            } else if (P[k] < lo[k] || P[k] > hi[k]) {
                tmax = -INFINITY;
            }
        }
        double tin = tmin > 0.0 ? tmin : 0.0;
        if (!(tmax > tin)) goto leak;
        for (int k = 0; k < 3; ++k) P[k] += tin * D[k];
        rec->track += tin;
        int ic[3], is[3];
        for (int k = 0; k < 3; ++k) {
            int a = (int)floor((P[k] - lo[k]) / dl[k]);
            ic[k] = a < 0 ? 0 : (a > n[k] - 1 ? n[k] - 1 : a);
            int b = (int)floor((P[k] - lo[k]) / dls[k]);
            is[k] = b < 0 ? 0 : (b > ns[k] - 1 ? ns[k] - 1 : b);
        }
        pt.R = orc_range(ORC_WATER, pt.E);
        for (;;) {
            if (++iter > ORC_MAX_ITER) goto fail;
            int64_t cidx = ic[0] + (int64_t)n[0] * (ic[1] + (int64_t)n[1] * ic[2]);
            double rho, spr;
            orc_hu_props(pb->curve, (double)pb->hu[cidx], &rho, &spr);
            orc_medium med = {ORC_WATER, spr * rc->sc->spr_scale, rho, ORC_MAT[ORC_WATER].za, ORC_MAT[ORC_WATER].X0};
            /* distance to the next voxel boundary of either grid */
            double dc[3], ds[3], svox = INFINITY;
            for (int k = 0; k < 3; ++k) {
                dc[k] = ds[k] = INFINITY;
                if (D[k] > 0.0) {
                    dc[k] = (lo[k] + (ic[k] + 1) * dl[k] - P[k]) / D[k];
                    ds[k] = (lo[k] + (is[k] + 1) * dls[k] - P[k]) / D[k];
                } else if (D[k] < 0.0) {
                    dc[k] = (lo[k] + ic[k] * dl[k] - P[k]) / D[k];
                    ds[k] = (lo[k] + is[k] * dls[k] - P[k]) / D[k];
                }
                if (dc[k] < 0.0) dc[k] = 0.0;
                if (ds[k] < 0.0) ds[k] = 0.0;
                if (dc[k] < svox) svox = dc[k];
                if (ds[k] < svox) svox = ds[k];
            }
            int64_t sidx = is[0] + (int64_t)ns[0] * (is[1] + (int64_t)ns[1] * is[2]);
            for (int k = 0; k < 3; ++k) { pt.p[k] = P[k]; pt.d[k] = D[k]; }
            ch_step(&med, &pt, svox, op, &st, &so);
            tl[7] += 1.0;
            rec->steps += 1;
            rec->path += so.s;
            rec->track += so.s;
            /* score the step's deposit in the voxel where the step starts */
            {
                if (rc->q) {
                    int64_t q = (int64_t)nearbyint(so.dE * (rc->mode == 0 ? sp->weight : 1.0) * fscale);
                    int64_t* dst = rc->mode == 0 ? &rc->q[sidx] : &rc->q[(int64_t)spot_index * rc->nvox + sidx];
#pragma omp atomic
                    *dst += q;
                }
                rec->e_dep += so.dE;
                rec->q_dep += (int64_t)nearbyint(so.dE * fscale);
                tl[1] += so.dE;
            }
            if (so.killed) {
                if (so.killed == 2) tl[5] += so.dE;
                if (so.killed == 2 && rho < ORC_LOW_RHO) rec->flags |= 4;
                rec->fate = so.killed == 2 ? FATE_NUC : FATE_STOP;
                for (int k = 0; k < 3; ++k) P[k] = pt.p[k];
                goto done;
            }
            if (so.limiter == LIM_GEOM) {
                int out = 0, crossed = -1;
                for (int k = 0; k < 3; ++k) {
                    int sgn = D[k] > 0.0 ? 1 : -1;
                    if (D[k] != 0.0 && dc[k] == svox) { ic[k] += sgn; crossed = k; }
                    if (D[k] != 0.0 && ds[k] == svox) is[k] += sgn;
                    if (ic[k] < 0 || ic[k] >= n[k] || is[k] < 0 || is[k] >= ns[k]) out = 1;
                }
                if (out) { for (int k = 0; k < 3; ++k) P[k] = pt.p[k]; goto leak; }
                if (crossed >= 0) {
                    double rho2, spr2;
                    orc_hu_props(pb->curve, (double)pb->hu[ic[0] + (int64_t)n[0] * (ic[1] + (int64_t)n[1] * ic[2])],
                                 &rho2, &spr2);
                    if (fabs(D[crossed]) < 0.01 * fabs(spr2 - spr)) rec->flags |= 8;
                }
            }
            /* lateral displacement, confined to the current voxel of both grids */
            for (int k = 0; k < 3; ++k) {
                double vlo = lo[k] + ic[k] * dl[k], vhi = lo[k] + (ic[k] + 1) * dl[k];
                double slo = lo[k] + is[k] * dls[k], shi = lo[k] + (is[k] + 1) * dls[k];
                if (slo > vlo) vlo = slo;
                if (shi < vhi) vhi = shi;
                double x = pt.p[k] + so.disp[k];
                P[k] = x < vlo ? vlo : (x > vhi ? vhi : x);
                D[k] = pt.d[k];
            }
        }
    }

leak:
    rec->fate = FATE_LEAK;
    rec->e_end = pt.E;
    tl[2] += pt.E;
    goto finish;
fail:
    rec->fate = FATE_ERR;
    rec->e_end = pt.E;
    tl[2] += pt.E;
    tl[8] += 1.0;
    goto finish;
done:
finish:
    if (in_patient) { for (int k = 0; k < 3; ++k) rec->pos[k] = P[k]; }
    else bev_to_patient(bm, rc->sc, pt.p, rec->pos);
}

/* ------------------------------------------------------------------ */
/* Driver: all histories of all given spots for one scenario.          */
/* ------------------------------------------------------------------ */
/* mode 0: q is one grid of the scoring grid's size, deposits weighted by
 *         the spot weight;  mode 1: q holds n_spots unweighted columns.
 * tally: ORC_NTALLY doubles (added to).  rec: optional per-history records
 * in spot order, history order; only the first rec_cap are written. */
/* Conditioning of a recorded history: the same history (same random
 * numbers) with its start moved by +-ORC_COND_MM along each BEV axis, scored
 * nowhere.  A rounding-level change of the path that moves the end point by
 * more than 1e-4 of the track (a face met at grazing incidence just before a
 * change of material, a crossing order that flips) sets bit 5; one that
 * changes the fate or the scored energy by more than 1e-4 sets bit 6. */
#define ORC_COND_MM 2e-5
static void condition_flags(const orc_run_ctx* rc, const orc_spot* sp, int spot_index, int64_t h, orc_record* r)
{
    orc_run_ctx dry = *rc;
    dry.q = NULL;
    static const double dirs[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
    for (int k = 0; k < 4; ++k) {
        double tl[ORC_NTALLY] = {0};
        double shift[2] = {ORC_COND_MM * dirs[k][0], ORC_COND_MM * dirs[k][1]};
        orc_record p;
        transport_history(&dry, sp, spot_index, h, &p, tl, shift);
        double track = r->track > 1.0 ? r->track : 1.0;
        double dx = p.pos[0] - r->pos[0], dy = p.pos[1] - r->pos[1], dz = p.pos[2] - r->pos[2];
        if (sqrt(dx * dx + dy * dy + dz * dz) > 1e-4 * track) r->flags |= 32;
        double escale = fabs(r->e_dep) > 1.0 ? fabs(r->e_dep) : 1.0;
        if (p.fate != r->fate || fabs(p.e_dep - r->e_dep) > 1e-4 * escale) r->flags |= 64;
    }
}

int orc_run(const orc_grid* ct, const int16_t* hu, const orc_curve* curve, const orc_grid* sg,
            const orc_beam* beams, const double* poly_xy,
            const orc_spot* spots, int n_spots, const orc_scen* sc, const orc_opts* op,
            int mode, int64_t* q, double* tally, orc_record* rec, int64_t rec_cap, int nthreads)
{
    orc_init_tables();
    orc_problem pb = {ct, hu, curve, sg, beams, poly_xy};
    orc_run_ctx rc = {&pb, sc, op, mode, q, (int64_t)sg->nx * sg->ny * sg->nz};
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (n_spots + 1));
    if (!off) return -1;
    off[0] = 0;
    for (int i = 0; i < n_spots; ++i) off[i + 1] = off[i] + spots[i].n_hist;
    int64_t total = off[n_spots];
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        double tl[ORC_NTALLY] = {0};
        orc_record tmp;
#pragma omp for schedule(dynamic, 16)
        for (int64_t gi = 0; gi < total; ++gi) {
            int lo = 0, hi = n_spots;           /* find spot: off[lo] <= gi < off[lo+1] */
            while (hi - lo > 1) { int mid = (lo + hi) / 2; if (off[mid] <= gi) lo = mid; else hi = mid; }
            const orc_spot* sp = &spots[lo];
            int64_t h = sp->h_begin + (gi - off[lo]);
            orc_record* r = (rec && gi < rec_cap) ? &rec[gi] : &tmp;
            transport_history(&rc, sp, lo, h, r, tl, NULL);
            if (r != &tmp) condition_flags(&rc, sp, lo, h, r);
        }
#pragma omp critical
        for (int i = 0; i < ORC_NTALLY; ++i) tally[i] += tl[i];
    }
    free(off);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Learned aperture surrogate: geometry features and training tracks.  */
/* ------------------------------------------------------------------ */
/* The surrogate is not part of the paper: it replaces condensed-history
 * stepping inside the brass block (Sec. 2.B) by one draw from a learned
 * distribution.  Its inputs, outputs and training tracks are defined here
 * from the plain aperture transport above; parity of the learned part is
 * pinned by that plain path (its dose), not by the paper. */
#define SUR_DCAP 12.0        /* mm: edge distance beyond which it is clipped     */
#define SUR_E_LO 40.0        /* MeV: training energies U(E_LO, E_HI)              */
#define SUR_E_HI 230.0
#define SUR_ANG_SIGMA 0.04   /* incidence direction cosines N(0, s^2) ...         */
#define SUR_ANG_MAX 0.12     /* ... clamped to +-ANG_MAX                           */
#define SUR_DIR_SCALE 0.05   /* exit direction change per target unit              */
#define SUR_SLOT_ENTRY 5u    /* Philox slot of the incidence angles                */

/* Signed curvature (1/mm) of polygon vertex i: turning angle over half the
 * two adjacent edge lengths, positive where the opening is locally convex. */
static double vertex_curvature(const double* poly, int n, int i, double orient)
{
    int a = (i + n - 1) % n, b = (i + 1) % n;
    double e0x = poly[2 * i] - poly[2 * a], e0y = poly[2 * i + 1] - poly[2 * a + 1];
    double e1x = poly[2 * b] - poly[2 * i], e1y = poly[2 * b + 1] - poly[2 * i + 1];
    double turn = atan2(e0x * e1y - e0y * e1x, e0x * e1x + e0y * e1y);
    double len = 0.5 * (sqrt(e0x * e0x + e0y * e0y) + sqrt(e1x * e1x + e1y * e1y));
    return orient * turn / len;
}

/* Nearest point of the polygon boundary to (x, y).  out = {distance,
 * nearest x, nearest y, curvature there}; the curvature is interpolated
 * linearly along the nearest edge between its vertices' curvatures, so it
 * does not depend on which of two equidistant edges is taken. */
void orc_nearest_edge(const double* poly, int n, double x, double y, double out[4])
{
    double area2 = 0.0;
    for (int i = 0; i < n; ++i) {
        int j = (i + 1) % n;
        area2 += poly[2 * i] * poly[2 * j + 1] - poly[2 * j] * poly[2 * i + 1];
    }
    double orient = area2 >= 0.0 ? 1.0 : -1.0;
    double best = INFINITY, bx = 0.0, by = 0.0;
    int bi = 0;
    double bt = 0.0;
    for (int i = 0; i < n; ++i) {
        int j = (i + 1) % n;
        double ax = poly[2 * i], ay = poly[2 * i + 1];
        double ex = poly[2 * j] - ax, ey = poly[2 * j + 1] - ay;
        double t = ((x - ax) * ex + (y - ay) * ey) / (ex * ex + ey * ey);
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
        double qx = ax + t * ex, qy = ay + t * ey;
        double d = sqrt((qx - x) * (qx - x) + (qy - y) * (qy - y));
        if (d < best) { best = d; bx = qx; by = qy; bi = i; bt = t; }
    }
    double k0 = vertex_curvature(poly, n, bi, orient);
    double k1 = vertex_curvature(poly, n, (bi + 1) % n, orient);
    out[0] = best;
    out[1] = bx;
    out[2] = by;
    out[3] = (1.0 - bt) * k0 + bt * k1;
}

/* Six surrogate inputs of a proton at (x, y) on the entrance plane of the
 * block with BEV direction d and energy E.  frame = {n_x, n_y, u_n, u_t}:
 * n is the unit vector from the nearest boundary point to the proton (into
 * the brass), t = (-n_y, n_x), u_n and u_t the direction's components. */
void orc_surrogate_features(const double* poly, int n, double thickness, double x, double y,
                            const double d[3], double E, double feat[6], double frame[4])
{
    double ne[4];
    orc_nearest_edge(poly, n, x, y, ne);
    double nx = (x - ne[1]) / ne[0], ny = (y - ne[2]) / ne[0];
    double un = d[0] * nx + d[1] * ny, ut = -d[0] * ny + d[1] * nx;
    double rmm = orc_range(ORC_BRASS, E) / ORC_MAT[ORC_BRASS].rho;
    double dc = ne[0] < SUR_DCAP ? ne[0] : SUR_DCAP;
    feat[0] = dc / (0.5 * SUR_DCAP) - 1.0;
    feat[1] = (E - 0.5 * (SUR_E_LO + SUR_E_HI)) / (0.5 * (SUR_E_HI - SUR_E_LO));
    feat[2] = un / SUR_ANG_SIGMA;
    feat[3] = ut / SUR_ANG_SIGMA;
    feat[4] = 8.0 * ne[3] - 1.0;
    feat[5] = rmm / thickness - 1.0;
    frame[0] = nx; frame[1] = ny; frame[2] = un; frame[3] = ut;
}

/* Training tracks: n_tracks histories per geometry g (beam g: aperture
 * only), each started on the block's entrance plane near the opening and
 * carried through the block by the plain transport.  Entry of history h of
 * geometry g, key (seed low, g ^ seed high):
 *   slot 0, step 0 -> u0..u2: E = E_LO + (E_HI - E_LO) u0; phi = 2 pi u1;
 *     d = d_hi u2^2 (denser near the edge, where the penumbra is made) with
 *     d_hi = min(DCAP, 1.2 R_brass(E)) when 1.2 R_brass(E)
 *     is below the block thickness, else DCAP; the proton starts at radius
 *     r_circ + d, angle phi, where r_circ is the largest vertex radius;
 *   slot 5, step 0 -> two normals z0, z1 (first Box-Muller pair):
 *     theta_n, theta_t = clamp(ANG_SIGMA z, +-ANG_MAX) along the radial and
 *     tangential unit vectors at phi; d_z = sqrt(1 - theta_n^2 - theta_t^2);
 *   slot 3, step 0 -> nuclear mean-free-path count, as for a source proton.
 * Outputs per track (index g * n_tracks + h): feat[6] (orc_surrogate_features
 * at the entry), label (1: left through the exit plane), target[5] for
 * label 1 (else zeros):
 *   y0 = 5 (E_in - E_out) / E_in,
 *   y1 = (exit - entry) . n - T u_n / w_in,  y2 = (exit - entry) . t - T u_t / w_in,
 *   y3 = (d_out . n - u_n) / DIR_SCALE,      y4 = (d_out . t - u_t) / DIR_SCALE,
 * and the plain transport's fate and ill-conditioning flags. */
int orc_surrogate_tracks(const orc_beam* beams, const double* poly_xy, int n_geom, int64_t n_tracks,
                         const orc_opts* op, double* feat, int32_t* label, double* target,
                         int32_t* fate, int32_t* flags, int nthreads)
{
    orc_init_tables();
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int64_t total = (int64_t)n_geom * n_tracks;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t gi = 0; gi < total; ++gi) {
        int g = (int)(gi / n_tracks);
        int64_t h = gi % n_tracks;
        const orc_beam* bm = &beams[g];
        const double* poly = poly_xy + 2 * (int64_t)bm->poly_offset;
        double T = bm->ap_thickness;
        double tup = -bm->ap_down_to_iso - T;
        orc_stream st;
        st.key[0] = (uint32_t)op->seed;
        st.key[1] = (uint32_t)(op->seed >> 32) ^ (uint32_t)g;
        st.hist = (uint32_t)h;
        double u[4], z[4];
        stream_block(&st, 0u, 0u, u);
        double E = SUR_E_LO + (SUR_E_HI - SUR_E_LO) * u[0];
        double phi = 2.0 * M_PI * u[1];
        double r12 = 1.2 * orc_range(ORC_BRASS, E) / ORC_MAT[ORC_BRASS].rho;
        double dhi = (r12 < T) ? (r12 < SUR_DCAP ? r12 : SUR_DCAP) : SUR_DCAP;
        double dd = dhi * u[2] * u[2];
        double rc = 0.0;
        for (int i = 0; i < bm->nvert; ++i) {
            double rr = sqrt(poly[2 * i] * poly[2 * i] + poly[2 * i + 1] * poly[2 * i + 1]);
            if (rr > rc) rc = rr;
        }
        double cph = cos(phi), sph = sin(phi);
        stream_normals4(&st, 0u, SUR_SLOT_ENTRY, z);
        double tn = SUR_ANG_SIGMA * z[0], tt = SUR_ANG_SIGMA * z[1];
        if (tn > SUR_ANG_MAX) tn = SUR_ANG_MAX;
        if (tn < -SUR_ANG_MAX) tn = -SUR_ANG_MAX;
        if (tt > SUR_ANG_MAX) tt = SUR_ANG_MAX;
        if (tt < -SUR_ANG_MAX) tt = -SUR_ANG_MAX;
        orc_particle pt;
        memset(&pt, 0, sizeof pt);
        pt.p[0] = (rc + dd) * cph;
        pt.p[1] = (rc + dd) * sph;
        pt.p[2] = tup;
        pt.d[0] = tn * cph - tt * sph;
        pt.d[1] = tn * sph + tt * cph;
        pt.d[2] = sqrt(1.0 - tn * tn - tt * tt);
        pt.E = E;
        if (op->nuclear) {
            double un[4];
            stream_block(&st, 0u, 3u, un);
            pt.nlam = -log(un[0]);
        } else {
            pt.nlam = INFINITY;
        }
        double* f = feat + 6 * gi;
        double fr[4];
        orc_surrogate_features(poly, bm->nvert, T, pt.p[0], pt.p[1], pt.d, E, f, fr);
        double x0 = pt.p[0], y0 = pt.p[1], w0 = pt.d[2];
        orc_record rec;
        memset(&rec, 0, sizeof rec);
        double tl[ORC_NTALLY] = {0};
        long iter = 0;
        int r = aperture_block(bm, poly, &pt, op, &st, &rec, tl, &iter);
        double* y = target + 5 * gi;
        for (int k = 0; k < 5; ++k) y[k] = 0.0;
        label[gi] = r == 0;
        fate[gi] = r == 0 ? -1 : r;
        flags[gi] = rec.flags;
        if (r == 0) {
            double nx = fr[0], ny = fr[1], un = fr[2], ut = fr[3];
            double dx = pt.p[0] - x0, dy = pt.p[1] - y0;
            y[0] = 5.0 * (E - pt.E) / E;
            y[1] = dx * nx + dy * ny - T * un / w0;
            y[2] = -dx * ny + dy * nx - T * ut / w0;
            y[3] = (pt.d[0] * nx + pt.d[1] * ny - un) / SUR_DIR_SCALE;
            y[4] = (-pt.d[0] * ny + pt.d[1] * nx - ut) / SUR_DIR_SCALE;
        }
    }
    return 0;
}

/* Number of threads the oracle's parallel loop uses. */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Scoring-voxel density and dose (dose to medium).                    */
/* ------------------------------------------------------------------ */
/* Volume-weighted mean density of the CT voxels overlapping each scoring
 * voxel (both grids share their origin and extent). */
void orc_scoring_density(const orc_grid* ct, const int16_t* hu, const orc_curve* curve,
                         const orc_grid* sg, double* rho_out)
{
    const int n[3] = {ct->nx, ct->ny, ct->nz};
    const double dl[3] = {ct->dx, ct->dy, ct->dz};
    const int ns[3] = {sg->nx, sg->ny, sg->nz};
    const double dls[3] = {sg->dx, sg->dy, sg->dz};
    for (int K = 0; K < ns[2]; ++K)
        for (int J = 0; J < ns[1]; ++J)
            for (int I = 0; I < ns[0]; ++I) {
                int S[3] = {I, J, K};
                int c0[3], c1[3];
                for (int k = 0; k < 3; ++k) {
                    double a = S[k] * dls[k], b = (S[k] + 1) * dls[k];
                    c0[k] = (int)floor(a / dl[k]);
                    c1[k] = (int)ceil(b / dl[k]);
                    if (c0[k] < 0) c0[k] = 0;
                    if (c1[k] > n[k]) c1[k] = n[k];
                }
                double acc = 0.0, vol = 0.0;
                for (int z = c0[2]; z < c1[2]; ++z)
                    for (int y = c0[1]; y < c1[1]; ++y)
                        for (int x = c0[0]; x < c1[0]; ++x) {
                            int C[3] = {x, y, z};
                            double ov = 1.0;
                            for (int k = 0; k < 3; ++k) {
                                double a = S[k] * dls[k], b = (S[k] + 1) * dls[k];
                                double c = C[k] * dl[k], d = (C[k] + 1) * dl[k];
                                double l = (b < d ? b : d) - (a > c ? a : c);
                                ov *= l > 0.0 ? l : 0.0;
                            }
                            if (ov <= 0.0) continue;
                            double rho, spr;
                            orc_hu_props(curve, (double)hu[x + (int64_t)n[0] * (y + (int64_t)n[1] * z)], &rho, &spr);
                            acc += ov * rho;
                            vol += ov;
                        }
                rho_out[I + (int64_t)ns[0] * (J + (int64_t)ns[1] * K)] = acc / vol;
            }
}

/* Dose (Gy) from fixed-point energy sums: q * 2^-F MeV / (rho * V). */
void orc_dose_from_q(const int64_t* q, int64_t nvox, const double* rho, double voxel_mm3,
                     int frac_bits, double* dose)
{
    double scale = ldexp(1.0, -frac_bits) * ORC_MEV_PER_G_TO_GY / (voxel_mm3 * 1e-3);
    for (int64_t i = 0; i < nvox; ++i) dose[i] = (double)q[i] * scale / rho[i];
}

/* ------------------------------------------------------------------ */
/* Global 3D gamma pass rate (paper Sec. 2.D, ref [80]).              */
/* ------------------------------------------------------------------ */
static double trilinear(const double* g, int nx, int ny, int nz, double fx, double fy, double fz, int* ok)
{
    if (fx < 0.0 || fy < 0.0 || fz < 0.0 || fx > nx - 1 || fy > ny - 1 || fz > nz - 1) { *ok = 0; return 0.0; }
    int x0 = (int)floor(fx), y0 = (int)floor(fy), z0 = (int)floor(fz);
    if (x0 > nx - 2) x0 = nx - 2 < 0 ? 0 : nx - 2;
    if (y0 > ny - 2) y0 = ny - 2 < 0 ? 0 : ny - 2;
    if (z0 > nz - 2) z0 = nz - 2 < 0 ? 0 : nz - 2;
    double ax = fx - x0, ay = fy - y0, az = fz - z0;
    int x1 = x0 + 1 < nx ? x0 + 1 : x0, y1 = y0 + 1 < ny ? y0 + 1 : y0, z1 = z0 + 1 < nz ? z0 + 1 : z0;
#define G(x, y, z) g[(x) + (int64_t)nx * ((y) + (int64_t)ny * (z))]
    double c00 = G(x0, y0, z0) * (1 - ax) + G(x1, y0, z0) * ax;
    double c10 = G(x0, y1, z0) * (1 - ax) + G(x1, y1, z0) * ax;
    double c01 = G(x0, y0, z1) * (1 - ax) + G(x1, y0, z1) * ax;
    double c11 = G(x0, y1, z1) * (1 - ax) + G(x1, y1, z1) * ax;
#undef G
    *ok = 1;
    double c0 = c00 * (1 - ay) + c10 * ay, c1 = c01 * (1 - ay) + c11 * ay;
    return c0 * (1 - az) + c1 * az;
}

/* Pass rate (%) of eval against ref: dose criterion dd_frac of the ref
 * maximum, distance dta_mm, evaluated on ref voxels >= thr_frac of the ref
 * maximum.  The eval dose is interpolated on a sub-grid of spacing 1/subdiv
 * voxel; since gamma <= 1 needs |r| <= dta, the search stops at dta. */
double orc_gamma_pass_rate(const double* ref, const double* eval, int nx, int ny, int nz,
                           double dx, double dy, double dz, double dd_frac, double dta_mm,
                           double thr_frac, int subdiv, int64_t* n_evaluated)
{
    int64_t nv = (int64_t)nx * ny * nz;
    double dmax = 0.0;
    for (int64_t i = 0; i < nv; ++i) if (ref[i] > dmax) dmax = ref[i];
    double dd = dd_frac * dmax, thr = thr_frac * dmax;
    int rx = (int)ceil(dta_mm / dx * subdiv), ry = (int)ceil(dta_mm / dy * subdiv), rz = (int)ceil(dta_mm / dz * subdiv);
    /* offsets within the DTA sphere, sorted by distance */
    int64_t cap = (int64_t)(2 * rx + 1) * (2 * ry + 1) * (2 * rz + 1);
    double* off = (double*)malloc(sizeof(double) * 4 * cap);
    int64_t m = 0;
    for (int k = -rz; k <= rz; ++k)
        for (int j = -ry; j <= ry; ++j)
            for (int i = -rx; i <= rx; ++i) {
                double ox = i * dx / subdiv, oy = j * dy / subdiv, oz = k * dz / subdiv;
                double r2 = ox * ox + oy * oy + oz * oz;
                if (r2 > dta_mm * dta_mm) continue;
                off[4 * m] = r2; off[4 * m + 1] = (double)i / subdiv; off[4 * m + 2] = (double)j / subdiv; off[4 * m + 3] = (double)k / subdiv;
                ++m;
            }
    /* insertion sort by r2 (small m) */
    for (int64_t a = 1; a < m; ++a) {
        double t[4] = {off[4 * a], off[4 * a + 1], off[4 * a + 2], off[4 * a + 3]};
        int64_t b = a - 1;
        while (b >= 0 && off[4 * b] > t[0]) { memcpy(&off[4 * (b + 1)], &off[4 * b], 4 * sizeof(double)); --b; }
        memcpy(&off[4 * (b + 1)], t, 4 * sizeof(double));
    }
    int64_t npass = 0, neval = 0;
#pragma omp parallel for reduction(+ : npass, neval) schedule(dynamic, 256)
    for (int64_t idx = 0; idx < nv; ++idx) {
        if (ref[idx] < thr || ref[idx] <= 0.0) continue;
        int x = (int)(idx % nx), y = (int)((idx / nx) % ny), z = (int)(idx / ((int64_t)nx * ny));
        ++neval;
        for (int64_t o = 0; o < m; ++o) {
            int ok;
            double de = trilinear(eval, nx, ny, nz, x + off[4 * o + 1], y + off[4 * o + 2], z + off[4 * o + 3], &ok);
            if (!ok) continue;
            double g2 = off[4 * o] / (dta_mm * dta_mm) + (de - ref[idx]) * (de - ref[idx]) / (dd * dd);
            if (g2 <= 1.0) { ++npass; break; }
        }
    }
    free(off);
    if (n_evaluated) *n_evaluated = neval;
    return neval ? 100.0 * (double)npass / (double)neval : 100.0;
}

/* ------------------------------------------------------------------ */
/* One condensed-history step from a fresh state, for unit tests.      */
/* ------------------------------------------------------------------ */
/* The particle starts at the origin moving along +z with energy E and the
 * medium's full residual range.  out[0..10] = s, dE, limiter, killed, E',
 * d'[3], disp[3]. */
void orc_step_sample(int table, double kappa, double rho, double za, double X0,
                     double E, double s_geom, int mcs, int straggling, int nuclear, double nlam,
                     uint64_t seed, int spot_key, uint32_t hist, uint32_t step, double* out)
{
    orc_init_tables();
    orc_medium med = {table, kappa, rho, za, X0};
    orc_opts op = {seed, mcs, straggling, nuclear, 24, 0};
    orc_stream st;
    st.key[0] = (uint32_t)seed;
    st.key[1] = (uint32_t)(seed >> 32) ^ (uint32_t)spot_key;
    st.hist = hist;
    orc_particle pt;
    memset(&pt, 0, sizeof pt);
    pt.d[2] = 1.0;
    pt.E = E;
    pt.nlam = nlam;
    pt.R = orc_range(table, E);
    pt.step = step;
    orc_step so;
    ch_step(&med, &pt, s_geom, &op, &st, &so);
    out[0] = so.s; out[1] = so.dE; out[2] = so.limiter; out[3] = so.killed; out[4] = pt.E;
    for (int k = 0; k < 3; ++k) { out[5 + k] = pt.d[k]; out[8 + k] = so.disp[k]; }
}

/*
 * avalanche_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, sequential, FP64 CPU restatement of microscopic electron
 * transport with avalanche multiplication: the AvalancheMicroscopic method
 * that "Accelerating Garfield++ with CUDA" (arXiv:2509.15377) moves to GPUs.
 * Only the test suite, the package's smoke check and the benchmark's CPU
 * baseline leg may load this file.  It shares no code, header, table or
 * constant with the CUDA library; both sides are written independently from
 * the paper and from the published definitions cited below.
 *
 * What the method computes (paper Sec. 2, Fig. 2):
 *   every electron of an avalanche is transported collision by collision
 *   ("electron transport"); an ionising collision adds a new electron to the
 *   stack ("stack processing"); the avalanche is complete when every electron
 *   carries a non-zero status code.  The paper does not spell out the
 *   transport physics; it relies on semi-classical Monte Carlo with the
 *   null-collision technique of Skullerud (Sec. 1, ref. HRSkullerud_1968) and
 *   tabulated per-level collision rates (Sec. 1, ref. Biagi).  The concrete
 *   step used here, in the order the loop below takes it:
 *     1. four uniforms from Philox4x32-10 keyed by the seed with the
 *        counter (flight index, 2 x avalanche, electron id);
 *     2. the field E (and uniform B) at the start of the flight, held
 *        constant for the flight;
 *     3. free flight dt = -ln(u0)/nu_max, truncated at the time limit, with
 *        the exact ballistic (E) or Lorentz (E and B) solution;
 *     4. kinetic energy from the velocity;
 *     5. boundary test ("Position is valid?", Fig. 2) -> non-zero status;
 *     6. linear interpolation of the cumulative per-level rates at the
 *        energy;
 *     7. real or null collision: R = u1*nu_max against the cumulative rates,
 *        a level whose threshold exceeds the energy counts as null;
 *     8. elastic (isotropic, recoil loss), excitation (threshold loss) or
 *        ionisation (threshold loss, uniform split of the remainder,
 *        isotropic secondary pushed to the stack, Fig. 2 "ionisation").
 *
 * Units: cm, ns, eV, V/cm, T.  Electron charge-to-mass ratio from CODATA
 * 2018, e/m = 1.75882001076e11 C/kg, which gives an acceleration of
 * 1.75882001076e-3 cm/ns^2 per V/cm and a cyclotron rate of 175.882001076
 * rad/ns per tesla.
 *
 * Pins (tests under tests/, marked "not gpu"):
 *   philox4x32_10 ...... published known-answer vectors (tests/golden).
 *   child_uid .......... SplitMix64 published output sequence (tests/golden)
 *                        and uniqueness over whole avalanches.
 *   flight ............. RK4 integration of the Lorentz force; the energy
 *                        ledger (kinetic energy change = field work).
 *   field .............. closed-form coaxial field; trilinear exact on affine
 *                        maps; the tetrahedral mesh: its elements tile the
 *                        box (volumes, one element per interior point),
 *                        linear interpolation exact on affine nodal values
 *                        and equal to the nodal value at a node, a mesh of a
 *                        constant field transports like the uniform field.
 *   table/selection .... brute-force level frequencies vs rate/nu_max.
 *   transport .......... drift velocity eE/(m nu) and the closed-form
 *                        transverse spread for a constant-rate elastic gas;
 *                        mean energy (1-r)^N for recoil-only cooling; Yule
 *                        (geometric) electron count with mean exp(nu_i T)
 *                        for a constant ionisation rate; Langevin E x B drift;
 *                        charge and energy conservation.
 *   ionisation split ... parity unpinned beyond the energy ledger (the paper
 *                        names no sharing model; the uniform split is a
 *                        reading, see the design notes).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread -lm.
 * Floating-point contraction is off so that every product and sum is the
 * one written here.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- units */
#define OR_ACCEL_PER_VCM 1.75882001076e-3 /* (e/m) * 1e-14: cm/ns^2 per V/cm */
#define OR_OMEGA_PER_T 175.882001076      /* (e/m) * 1e-9: rad/ns per T      */
#define OR_PI 3.14159265358979323846

/* electron status codes (non-zero = transport finished, paper Sec. 2) */
enum {
    OR_ACTIVE = 0,
    OR_ANODE = 1,        /* plate: z >= gap */
    OR_CATHODE = 2,      /* plate: z < 0 */
    OR_WIRE = 3,         /* coax / grid: r <= wire radius */
    OR_TUBE = 4,         /* coax: r >= tube radius */
    OR_OUT_OF_MAP = 5,   /* grid: outside the map box; mesh: in no element */
    OR_TIME = 6,         /* time limit reached */
    OR_COLL_LIMIT = 7,   /* real-collision limit reached */
    OR_FLIGHT_LIMIT = 8, /* 2^32-1 flights (counter exhausted) */
    OR_ATTACHED = 9      /* captured by an attachment collision */
};

/* level types: Fig. 2 "Collision is ionisation or attachment?" */
enum { OR_ELASTIC = 0, OR_EXCITATION = 1, OR_IONISATION = 2, OR_ATTACHMENT = 3 };
enum { OR_UNIFORM = 0, OR_PLATE = 1, OR_COAX = 2, OR_GRID = 3, OR_MESH = 4 };

typedef struct {
    int32_t n_levels;
    int32_t n_nodes;
    double d_eps;              /* eV between table nodes; node k at k*d_eps */
    const int32_t *level_type; /* [n_levels] */
    const double *threshold;   /* [n_levels] eV (energy lost) */
    const double *rate;        /* [n_nodes][n_levels], 1/ns */
    double recoil;             /* 2m/M for elastic recoil loss; 0 = none */
    double nu_max;             /* 1/ns; 0 = (1+1e-6) * max total rate */
    const double *xi0;         /* [n_levels] constant anisotropy, or NULL (all 0) */
    const double *screen;      /* [n_levels] screening energy (eV), or NULL (all 0) */
    double split_w;            /* ionisation sharing width (eV); 0 = uniform split */
} or_gas;

typedef struct {
    int32_t kind;
    double e0;                 /* UNIFORM/PLATE: E = (0,0,-e0) V/cm */
    double gap;                /* PLATE: anode at z = gap (cm) */
    double wire_r, tube_r, voltage; /* COAX (and GRID wire test) */
    double b[3];               /* uniform magnetic field, T */
    int32_t nx, ny, nz;        /* GRID nodes */
    double origin[3], spacing[3];
    const float *grid;         /* GRID: host float4 (Ex,Ey,Ez,-) per node, x fastest */
    int64_t n_mesh_nodes, n_tets;  /* MESH: nodes and tetrahedra */
    const double *mesh_nodes;  /* MESH: [n_mesh_nodes][3] node positions (cm) */
    const int32_t *mesh_tets;  /* MESH: [n_tets][4] node indices */
    const float *mesh_values;  /* MESH: [n_mesh_nodes][4] (Ex, Ey, Ez, weighting potential) */
} or_field;

typedef struct {
    int64_t n_primaries;
    int32_t n_avalanches;
    const double *x, *y, *z, *t, *e; /* primary position, time, energy */
    const double *dx, *dy, *dz;      /* primary unit direction */
    const int32_t *aval;             /* avalanche of each primary */
    const uint64_t *uid;             /* electron id of each primary */
    const double *aval_field;        /* PLATE: per-avalanche |E| or NULL */
    uint64_t seed;
    double t_max;                    /* ns; <= 0 means none */
    uint32_t coll_limit;             /* real collisions; 0 means none */
    int32_t n_threads;
    int32_t majorant;                /* 0: one global nu_max; 1: banded (below) */
    double window;                   /* banded: flight window = window / band rate */
    double band_width;               /* banded: eV per energy band (whole nodes) */
    int32_t substeps;                /* field evaluations per flight (<= 1: one, held) */
    int32_t crossing;                /* 1: an electron leaving the volume ends at the
                                        first crossing of the boundary */
    int32_t signal_kind;             /* readout electrode (OR_W_*), 0: no signal */
    int32_t signal_bins;             /* time bins of the induced signal */
    double signal_t0, signal_dt;     /* bin j covers [t0 + j dt, t0 + (j+1) dt) */
    int32_t aval_base;               /* number of avalanche 0 in a larger workload: the
                                        random counters hold aval + aval_base, so
                                        avalanches [a0, a1) of a workload run alone with
                                        aval_base = a0 are those of the whole run (they
                                        are independent, Sec. 2) */
} or_run_args;

/* ------------------------------------------------ Philox4x32-10
 * J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11.  One round maps the counter
 * (c0,c1,c2,c3) with the round key (k0,k1) to
 *   (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)),
 * the key is advanced by the Weyl constants between rounds, ten rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Open-interval uniform from one 32-bit word: (w + 1/2) / 2^32, exact. */
static double uniform01(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* The four uniforms of draw `sub` (0 or 1) of flight `flight` of electron
 * `uid` in avalanche `aval`: the key is the seed alone, and the counter
 * (flight, 2 aval + sub, uid_lo, uid_hi) is distinct for every draw of the
 * run, so every draw is its own block of one Philox stream. */
static void draw4(uint64_t seed, int32_t aval, uint64_t uid, uint32_t flight,
                  uint32_t sub, double u[4])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {flight, ((uint32_t)aval << 1) | sub, (uint32_t)uid,
                       (uint32_t)(uid >> 32)};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    for (int i = 0; i < 4; ++i) u[i] = uniform01(w[i]);
}

/* ------------------------------------------------ SplitMix64 output function
 * G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014: z ^= z>>30; z *= 0xbf58476d1ce4e5b9;
 * z ^= z>>27; z *= 0x94d049bb133111eb; z ^= z>>31. */
uint64_t or_splitmix64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Id of the electron created by ionisation in flight `flight` of `parent`:
 * the SplitMix64 output of parent + golden * (flight + 1). */
uint64_t or_child_uid(uint64_t parent, uint32_t flight)
{
    return or_splitmix64_mix(parent + 0x9E3779B97F4A7C15ull * ((uint64_t)flight + 1u));
}

/* ------------------------------------------------ field (paper Fig. 2,
 * "Find E field"): E in V/cm at r.  Returns 0, or -1 if the grid is
 * queried outside its box (the caller's boundary test runs first). */
static void grid_node(const or_field *f, int i, int j, int k, double e[3])
{
    const float *p = f->grid + 4 * (((int64_t)k * f->ny + j) * f->nx + i);
    e[0] = p[0]; e[1] = p[1]; e[2] = p[2];
}

/* Field maps on a tetrahedral mesh (Sec. 3.1: the field maps are finite-element
 * solutions on tetrahedral meshes; a point's element is searched, then the
 * element's nodal values are interpolated).  The element of r is the
 * lowest-index closed tetrahedron (every barycentric coordinate >= 0) that
 * contains it, found by trying every element; the barycentric coordinates
 * come from Cramer's rule on the edge vectors from the element's first
 * node.  Returns the element, or -1 when r is in none. */
static double triple(const double a[3], const double b[3], const double c[3])
{
    return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
           a[2] * (b[0] * c[1] - b[1] * c[0]);
}

int64_t or_mesh_locate(const or_field *f, const double r[3], double lam[4])
{
    for (int64_t t = 0; t < f->n_tets; ++t) {
        const int32_t *q = f->mesh_tets + 4 * t;
        const double *v[4];
        for (int i = 0; i < 4; ++i) v[i] = f->mesh_nodes + 3 * (int64_t)q[i];
        int out = 0;
        for (int d = 0; d < 3 && !out; ++d) {
            double lo = v[0][d], hi = v[0][d];
            for (int i = 1; i < 4; ++i) {
                if (v[i][d] < lo) lo = v[i][d];
                if (v[i][d] > hi) hi = v[i][d];
            }
            out = r[d] < lo || r[d] > hi;
        }
        if (out) continue;
        double e1[3], e2[3], e3[3], dr[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = v[1][d] - v[0][d];
            e2[d] = v[2][d] - v[0][d];
            e3[d] = v[3][d] - v[0][d];
            dr[d] = r[d] - v[0][d];
        }
        const double det = triple(e1, e2, e3);
        const double l1 = triple(dr, e2, e3) / det;
        const double l2 = triple(e1, dr, e3) / det;
        const double l3 = triple(e1, e2, dr) / det;
        const double l0 = 1.0 - l1 - l2 - l3;
        if (l0 >= 0.0 && l1 >= 0.0 && l2 >= 0.0 && l3 >= 0.0) {
            lam[0] = l0; lam[1] = l1; lam[2] = l2; lam[3] = l3;
            return t;
        }
    }
    return -1;
}

/* Component c of the mesh's nodal values interpolated at r in element t. */
static double mesh_interp(const or_field *f, int64_t t, const double lam[4], int c)
{
    const int32_t *q = f->mesh_tets + 4 * t;
    double x = 0.0;
    for (int i = 0; i < 4; ++i) x += lam[i] * (double)f->mesh_values[4 * (int64_t)q[i] + c];
    return x;
}

void or_field_eval(const or_field *f, double plate_e, const double r[3], double e[3])
{
    e[0] = e[1] = e[2] = 0.0;
    if (f->kind == OR_UNIFORM) {
        e[2] = -f->e0;
    } else if (f->kind == OR_PLATE) {
        e[2] = -plate_e;
    } else if (f->kind == OR_COAX) {
        /* E = V / (r ln(b/a)) along r-hat in the transverse plane */
        double r2 = r[0] * r[0] + r[1] * r[1];
        double s = f->voltage / (log(f->tube_r / f->wire_r) * r2);
        e[0] = s * r[0];
        e[1] = s * r[1];
    } else if (f->kind == OR_MESH) { /* linear interpolation in the element */
        double lam[4];
        const int64_t t = or_mesh_locate(f, r, lam);
        if (t >= 0)
            for (int c = 0; c < 3; ++c) e[c] = mesh_interp(f, t, lam, c);
    } else { /* OR_GRID: trilinear interpolation of the node values */
        int n[3] = {f->nx, f->ny, f->nz};
        int idx[3];
        double w[3];
        for (int d = 0; d < 3; ++d) {
            double g = (r[d] - f->origin[d]) / f->spacing[d];
            int i = (int)floor(g);
            if (i < 0) i = 0;
            if (i > n[d] - 2) i = n[d] - 2;
            idx[d] = i;
            w[d] = g - i;
        }
        for (int c = 0; c < 8; ++c) {
            int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
            double wt = (di ? w[0] : 1.0 - w[0]) * (dj ? w[1] : 1.0 - w[1]) *
                        (dk ? w[2] : 1.0 - w[2]);
            double en[3];
            grid_node(f, idx[0] + di, idx[1] + dj, idx[2] + dk, en);
            e[0] += wt * en[0];
            e[1] += wt * en[1];
            e[2] += wt * en[2];
        }
    }
}

/* ------------------------------------------------ boundary test
 * ("Position is valid?", Fig. 2): 0 inside, else the status code. */
int or_boundary(const or_field *f, const double r[3])
{
    if (f->kind == OR_PLATE) {
        if (r[2] >= f->gap) return OR_ANODE;
        if (r[2] < 0.0) return OR_CATHODE;
    } else if (f->kind == OR_COAX) {
        double r2 = r[0] * r[0] + r[1] * r[1];
        if (r2 <= f->wire_r * f->wire_r) return OR_WIRE;
        if (r2 >= f->tube_r * f->tube_r) return OR_TUBE;
    } else if (f->kind == OR_GRID) {
        double r2 = r[0] * r[0] + r[1] * r[1];
        if (f->wire_r > 0.0 && r2 <= f->wire_r * f->wire_r) return OR_WIRE;
        int n[3] = {f->nx, f->ny, f->nz};
        for (int d = 0; d < 3; ++d) {
            double hi = f->origin[d] + (n[d] - 1) * f->spacing[d];
            if (r[d] < f->origin[d] || r[d] > hi) return OR_OUT_OF_MAP;
        }
    } else if (f->kind == OR_MESH) {
        double r2 = r[0] * r[0] + r[1] * r[1];
        if (f->wire_r > 0.0 && r2 <= f->wire_r * f->wire_r) return OR_WIRE;
        double lam[4];
        if (or_mesh_locate(f, r, lam) < 0) return OR_OUT_OF_MAP;
    }
    return 0;
}

/* ------------------------------------------------ free flight
 * Exact motion over dt under constant acceleration a (cm/ns^2) and a
 * uniform magnetic rotation vector w (rad/ns): dv/dt = a + v x w.
 * With w = 0 this is r += v dt + a dt^2/2, v += a dt.  Otherwise the part
 * along w-hat accelerates uniformly, the perpendicular part is the drift
 * (a x w)/|w|^2 plus a rotation of the rest about w-hat by -|w| dt. */
static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

void or_flight(double r[3], double v[3], const double a[3], const double w[3], double dt)
{
    double wn = sqrt(dot3(w, w));
    if (wn == 0.0) {
        for (int d = 0; d < 3; ++d) {
            r[d] = r[d] + v[d] * dt + 0.5 * a[d] * dt * dt;
            v[d] = v[d] + a[d] * dt;
        }
        return;
    }
    double bh[3] = {w[0] / wn, w[1] / wn, w[2] / wn};
    double vpar = dot3(v, bh), apar = dot3(a, bh);
    double axw[3];
    cross3(a, w, axw);
    double drift[3] = {axw[0] / (wn * wn), axw[1] / (wn * wn), axw[2] / (wn * wn)};
    double u[3], bxu[3];
    for (int d = 0; d < 3; ++d) u[d] = v[d] - vpar * bh[d] - drift[d];
    cross3(bh, u, bxu);
    double th = wn * dt, c = cos(th), s = sin(th);
    for (int d = 0; d < 3; ++d) {
        r[d] = r[d] + (vpar * dt + 0.5 * apar * dt * dt) * bh[d] + drift[d] * dt +
               u[d] * (s / wn) - bxu[d] * ((1.0 - c) / wn);
        v[d] = (vpar + apar * dt) * bh[d] + drift[d] + u[d] * c - bxu[d] * s;
    }
}

/* ------------------------------------------------ boundary crossings
 * The first time in (0, hi] at which the flight from (r0, v0) under the
 * held acceleration acc (and rotation w) is outside the volume, given that
 * it is outside at hi: bisection to within hi * 2^-60; the state at the
 * returned time is outside. */
static double first_exit(const or_field *f, const double r0[3], const double v0[3],
                         const double acc[3], const double w[3], double hi)
{
    double lo = 0.0;
    for (int it = 0; it < 60; ++it) {
        double mid = 0.5 * (lo + hi);
        double r[3] = {r0[0], r0[1], r0[2]}, v[3] = {v0[0], v0[1], v0[2]};
        or_flight(r, v, acc, w, mid);
        if (or_boundary(f, r))
            hi = mid;
        else
            lo = mid;
    }
    return hi;
}

/* Plate without B: z(t) = z0 + vz t + az t^2 / 2 is a parabola, so a step
 * that starts and ends inside may still have left the gap at its vertex.
 * Returns the status at the vertex if the vertex lies inside (0, h) and
 * outside the gap, with *t_out the vertex time; else 0. */
static int plate_vertex_exit(const or_field *f, const double r0[3], const double v0[3],
                             const double acc[3], double h, double *t_out)
{
    if (acc[2] == 0.0) return 0;
    double tv = -v0[2] / acc[2];
    if (!(tv > 0.0 && tv < h)) return 0;
    double r[3] = {r0[0] + v0[0] * tv + 0.5 * acc[0] * tv * tv,
                   r0[1] + v0[1] * tv + 0.5 * acc[1] * tv * tv,
                   r0[2] + v0[2] * tv + 0.5 * acc[2] * tv * tv};
    int st = or_boundary(f, r);
    if (st) *t_out = tv;
    return st;
}

/* Largest field magnitude of the volume (V/cm): the bound of the banded
 * majorant when the field is re-evaluated along a flight.  0 for fields
 * that are the same everywhere (the held-field bound stays exact). */
static double field_emax(const or_field *f)
{
    if (f->kind == OR_COAX) return fabs(f->voltage) / (log(f->tube_r / f->wire_r) * f->wire_r);
    if (f->kind == OR_GRID) {
        double m = 0.0;
        int64_t n = (int64_t)f->nx * f->ny * f->nz;
        for (int64_t i = 0; i < n; ++i) {
            const float *p = f->grid + 4 * i;
            double e = sqrt((double)p[0] * p[0] + (double)p[1] * p[1] + (double)p[2] * p[2]);
            if (e > m) m = e;
        }
        return m;
    }
    if (f->kind == OR_MESH) { /* |E| is convex in an element: its largest value is at a node */
        double m = 0.0;
        for (int64_t i = 0; i < f->n_mesh_nodes; ++i) {
            const float *p = f->mesh_values + 4 * i;
            double e = sqrt((double)p[0] * p[0] + (double)p[1] * p[1] + (double)p[2] * p[2]);
            if (e > m) m = e;
        }
        return m;
    }
    return 0.0;
}

/* ------------------------------------------------ induced signal
 * Shockley-Ramo: a charge q at r induces -q phi_w(r) on the readout
 * electrode, phi_w the electrode's weighting potential (1 on the electrode,
 * 0 on the others).  An electron (q = -e) moving from r_a to r_b therefore
 * induces phi_w(r_b) - phi_w(r_a) in units of e, whatever its path; the
 * signal in a time bin is that difference between the electron's positions
 * at the bin's edges (or its birth and end inside the bin). */
enum { OR_W_NONE = 0, OR_W_PLATE = 1, OR_W_COAX = 2, OR_W_MAP = 3 };

static double weighting_potential(const or_field *f, int kind, const double r[3])
{
    if (kind == OR_W_PLATE) return r[2] / f->gap; /* anode at z = gap */
    if (kind == OR_W_COAX) {                        /* wire at r = a, tube at r = b */
        double rr = sqrt(r[0] * r[0] + r[1] * r[1]);
        return log(rr / f->tube_r) / log(f->wire_r / f->tube_r);
    }
    if (kind == OR_W_MAP && f->kind == OR_MESH) { /* linear in the element */
        double lam[4];
        const int64_t t = or_mesh_locate(f, r, lam);
        return t >= 0 ? mesh_interp(f, t, lam, 3) : 0.0;
    }
    if (kind == OR_W_MAP) { /* trilinear interpolation of the nodes' 4th component */
        int n[3] = {f->nx, f->ny, f->nz};
        int idx[3];
        double w[3];
        for (int d = 0; d < 3; ++d) {
            double g = (r[d] - f->origin[d]) / f->spacing[d];
            int i = (int)floor(g);
            if (i < 0) i = 0;
            if (i > n[d] - 2) i = n[d] - 2;
            idx[d] = i;
            w[d] = g - i;
        }
        double phi = 0.0;
        for (int c = 0; c < 8; ++c) {
            int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
            double wt = (di ? w[0] : 1.0 - w[0]) * (dj ? w[1] : 1.0 - w[1]) *
                        (dk ? w[2] : 1.0 - w[2]);
            const float *p = f->grid + 4 * (((int64_t)(idx[2] + dk) * f->ny + (idx[1] + dj)) *
                                                f->nx + (idx[0] + di));
            phi += wt * p[3];
        }
        return phi;
    }
    return 0.0;
}

/* Test hook: the weighting potential above. */
double or_weighting_potential(const or_field *f, int kind, const double r[3])
{
    return weighting_potential(f, kind, r);
}

/* Per-electron signal state: the next bin edge and the potential at the
 * last edge (or birth). */
typedef struct {
    int64_t next;     /* index of the next bin edge t0 + next dt after the current time */
    double phi_last;
} or_signal;

static void signal_start(const or_run_args *a, const or_field *f, or_signal *sg, double t,
                         const double r[3])
{
    double x = (t - a->signal_t0) / a->signal_dt;
    sg->next = x < 0.0 ? 0 : (int64_t)floor(x) + 1;
    sg->phi_last = sg->next >= 1 ? weighting_potential(f, a->signal_kind, r) : 0.0;
}

/* A step from (r0, v0) at time ts to te under acc (and rotation w): every
 * bin edge it passes closes a bin. */
static void signal_step(const or_run_args *a, const or_field *f, or_signal *sg, double *sig,
                        const double r0[3], const double v0[3], const double acc[3],
                        const double w[3], double ts, double te)
{
    for (;;) {
        if (sg->next > a->signal_bins) return;
        double tb = a->signal_t0 + (double)sg->next * a->signal_dt;
        if (tb > te) return;
        double r[3] = {r0[0], r0[1], r0[2]}, v[3] = {v0[0], v0[1], v0[2]};
        or_flight(r, v, acc, w, tb - ts);
        double ph = weighting_potential(f, a->signal_kind, r);
        if (sg->next >= 1) sig[sg->next - 1] += ph - sg->phi_last;
        sg->phi_last = ph;
        sg->next += 1;
    }
}

static void signal_end(const or_run_args *a, const or_field *f, const or_signal *sg, double *sig,
                       const double r[3])
{
    if (sg->next >= 1 && sg->next <= a->signal_bins)
        sig[sg->next - 1] += weighting_potential(f, a->signal_kind, r) - sg->phi_last;
}

/* ------------------------------------------------ rate table */
typedef struct {
    int L, N;
    double d_eps, nu_max, recoil;
    int type[64];
    double thr[64];
    double xi0[64], screen[64]; /* angular model per level (see level_xi) */
    double split_w;
    double *cum; /* [N][L]: running sum over levels 0..j of the rate */
    double top;  /* largest total rate over the nodes */
    int band_nodes, B; /* banded majorant: nodes per band, number of bands */
    double *bmax;      /* [B]: largest total rate over the band's nodes */
    double field_emax; /* > 0: bound |E| by this in the banded majorant (a field
                          re-evaluated along the flight), 0: the held field */
} or_table;

static int table_build(const or_gas *g, or_table *t)
{
    if (g->n_levels < 1 || g->n_levels > 64 || g->n_nodes < 2 || !(g->d_eps > 0.0)) return -1;
    t->L = g->n_levels;
    t->N = g->n_nodes;
    t->d_eps = g->d_eps;
    t->recoil = g->recoil;
    for (int j = 0; j < t->L; ++j) {
        t->type[j] = g->level_type[j];
        t->thr[j] = g->threshold[j];
        t->xi0[j] = g->xi0 ? g->xi0[j] : 0.0;
        t->screen[j] = g->screen ? g->screen[j] : 0.0;
        if (t->type[j] < OR_ELASTIC || t->type[j] > OR_ATTACHMENT) return -1;
        if (!(t->xi0[j] > -1.0 && t->xi0[j] < 1.0) || !(t->screen[j] >= 0.0)) return -1;
    }
    t->split_w = g->split_w;
    if (!(t->split_w >= 0.0)) return -1;
    t->cum = (double *)malloc(sizeof(double) * (size_t)t->N * t->L);
    if (!t->cum) return -1;
    double top = 0.0;
    for (int k = 0; k < t->N; ++k) {
        double s = 0.0;
        for (int j = 0; j < t->L; ++j) {
            s += g->rate[(int64_t)k * t->L + j];
            t->cum[(int64_t)k * t->L + j] = s;
        }
        if (s > top) top = s;
    }
    t->nu_max = g->nu_max > 0.0 ? g->nu_max : top * (1.0 + 1e-6);
    t->band_nodes = 0;
    t->B = 0;
    t->bmax = NULL;
    t->top = top;
    if (!(t->nu_max > 0.0) || t->nu_max < top) {
        free(t->cum);
        return -1;
    }
    return 0;
}

/* Energy bands for the banded majorant: band b spans the nodes
 * b*n .. (b+1)*n (n = band_width / d_eps, at least 1); since the rates are
 * linear between nodes, the largest total rate over the band's energies is
 * the largest node value.  Energies beyond the last node belong to the
 * last band (their rate is the last node's).  A band whose rates are all
 * zero gets the bound top * 2^-40 instead, so that its window stays
 * finite (any positive bound of a zero rate is exact). */
static int bands_build(or_table *t, double band_width)
{
    int n = (int)floor(band_width / t->d_eps + 0.5);
    if (n < 1) n = 1;
    int B = (t->N - 1 + n - 1) / n;
    if (B < 1) B = 1;
    t->bmax = (double *)malloc(sizeof(double) * (size_t)B);
    if (!t->bmax) return -1;
    for (int b = 0; b < B; ++b) {
        double m = 0.0;
        for (int k = b * n; k <= (b + 1) * n && k < t->N; ++k) {
            double c = t->cum[(int64_t)k * t->L + t->L - 1];
            if (c > m) m = c;
        }
        t->bmax[b] = m > 0.0 ? m : ldexp(t->top, -40);
    }
    t->band_nodes = n;
    t->B = B;
    return 0;
}

static int band_of(const or_table *t, double eps)
{
    double x = eps / (t->band_nodes * t->d_eps);
    if (!(x > 0.0)) return 0;
    if (x >= (double)t->B) return t->B - 1;
    int b = (int)floor(x);
    return b < t->B ? b : t->B - 1;
}

/* Banded majorant of one flight with velocity v in the held field E.
 * The window is tau = window / (bound of the current band).  Within it the
 * energy stays in a range [lo, hi]:
 *   no magnetic field: the flight is v + a t, so the energy is
 *     eps(t) = eps0 + g(t),  g(t) = -(v.E) t + (a1 |E|^2 / 2) t^2
 *   (the field's work, a convex parabola in t): hi = eps0 + max(g(tau), 0);
 *   lo = eps0 when v.E <= 0 (g rises from 0), else the vertex value
 *   eps0 - (v.E) t* / 2 at t* = (v.E) / (a1 |E|^2) if t* < tau, or
 *   eps0 + g(tau);
 *   with a magnetic field: |dv/dt| <= a1 |E| along the flight, so the
 *   displacement stays below |v| tau + a1 |E| tau^2 / 2 and
 *   [lo, hi] = eps0 -+ |E| (|v| tau + a1 |E| tau^2 / 2).
 * The majorant is the largest bound of the bands covering [lo, hi]; it
 * bounds the true rate along the flight because the table is linear
 * between nodes.  Returns it and sets *tau. */
static double kinetic_energy(const double v[3]);

static double banded_majorant(const or_table *tb, const double v[3], const double E[3], int has_b,
                              double window, double *tau)
{
    double eps0 = kinetic_energy(v);
    double w = window / tb->bmax[band_of(tb, eps0)];
    double lo, hi;
    if (tb->field_emax > 0.0) {
        /* the field changes along the flight: the reach of the largest
         * field magnitude (|dv/dt| <= a1 E_max) bounds the energy change */
        double Em = tb->field_emax;
        double D = Em * (sqrt(dot3(v, v)) * w + 0.5 * (OR_ACCEL_PER_VCM * Em) * w * w);
        lo = eps0 - D;
        hi = eps0 + D;
    } else if (!has_b) {
        double vE = dot3(v, E), E2 = dot3(E, E);
        double gw = -vE * w + 0.5 * OR_ACCEL_PER_VCM * E2 * w * w;
        hi = eps0 + (gw > 0.0 ? gw : 0.0);
        if (vE <= 0.0) {
            lo = eps0;
        } else {
            double ts = vE / (OR_ACCEL_PER_VCM * E2);
            lo = ts < w ? eps0 - 0.5 * vE * ts : eps0 + gw;
        }
    } else {
        double Em = sqrt(dot3(E, E));
        double D = Em * (sqrt(dot3(v, v)) * w + 0.5 * (OR_ACCEL_PER_VCM * Em) * w * w);
        lo = eps0 - D;
        hi = eps0 + D;
    }
    int b0 = band_of(tb, lo), b1 = band_of(tb, hi);
    double nu = 0.0;
    for (int b = b0; b <= b1; ++b)
        if (tb->bmax[b] > nu) nu = tb->bmax[b];
    *tau = w;
    return nu;
}

/* Test hook: the banded majorant above for a given gas and band width.
 * Returns the rate (1/ns), or a negative value for a bad table. */
double or_majorant(const or_gas *g, double band_width, const double v[3], const double E[3],
                   int has_b, double window, double *tau_out)
{
    or_table t;
    if (table_build(g, &t)) return -1.0;
    if (bands_build(&t, band_width)) {
        free(t.cum);
        return -1.0;
    }
    double tau = 0.0;
    t.field_emax = 0.0;
    double nu = banded_majorant(&t, v, E, has_b, window, &tau);
    if (tau_out) *tau_out = tau;
    free(t.cum);
    free(t.bmax);
    return nu;
}

/* Test hook: the largest field magnitude of a field (V/cm), the bound a run
 * with sub-steps gives the banded majorant (0 for fields that are the same
 * everywhere). */
double or_field_emax(const or_field *f) { return field_emax(f); }

/* Test hook: the banded majorant of a flight along which the field is
 * re-evaluated, with the field magnitude bounded by `emax` (> 0; as a run
 * with sub-steps sets it from or_field_emax).  Returns the rate (1/ns), or a
 * negative value for a bad table or emax <= 0. */
double or_majorant_reach(const or_gas *g, double band_width, const double v[3], double emax,
                         double window, double *tau_out)
{
    if (!(emax > 0.0)) return -1.0;
    or_table t;
    if (table_build(g, &t)) return -1.0;
    if (bands_build(&t, band_width)) {
        free(t.cum);
        return -1.0;
    }
    const double E0[3] = {0.0, 0.0, 0.0};
    double tau = 0.0;
    t.field_emax = emax;
    double nu = banded_majorant(&t, v, E0, 0, window, &tau);
    if (tau_out) *tau_out = tau;
    free(t.cum);
    free(t.bmax);
    return nu;
}

/* Cumulative rates at energy eps by linear interpolation between nodes;
 * energies at or beyond the last node use the last node. */
static void table_interp(const or_table *t, double eps, double *c)
{
    double x = eps / t->d_eps;
    int k;
    double f;
    if (x >= (double)(t->N - 1)) {
        k = t->N - 2;
        f = 1.0;
    } else {
        k = (int)floor(x);
        f = x - k;
    }
    const double *c0 = t->cum + (int64_t)k * t->L;
    const double *c1 = c0 + t->L;
    for (int j = 0; j < t->L; ++j) c[j] = c0[j] + f * (c1[j] - c0[j]);
}

/* Real or null collision (Fig. 2 "Collision?") for a flight drawn with the
 * majorant nu: level index, or -1 for null. */
static int table_select(const or_table *t, double eps, double u1, double nu)
{
    double c[64];
    table_interp(t, eps, c);
    double R = u1 * nu;
    for (int j = 0; j < t->L; ++j) {
        if (R < c[j]) {
            if (t->type[j] != OR_ELASTIC && eps < t->thr[j]) return -1;
            return j;
        }
    }
    return -1;
}

/* Test hook: the selection above for a given gas, energy and uniform. */
int or_select(const or_gas *g, double eps, double u1, double *nu_max_out)
{
    or_table t;
    if (table_build(g, &t)) return -2;
    int j = table_select(&t, eps, u1, t.nu_max);
    if (nu_max_out) *nu_max_out = t.nu_max;
    free(t.cum);
    return j;
}

/* ------------------------------------------------ per-avalanche storage */
typedef struct {
    double x0, y0, z0, t0, e0, x1, y1, z1, t1, e1;
    int32_t status;
    uint32_t n_flight;
    uint64_t uid;
    double ledger[4]; /* field work, inelastic loss, recoil loss, secondary share */
} or_endpoint;

typedef struct {
    double r[3], v[3], t, e0;
    uint64_t uid;
} or_pending;

typedef struct {
    or_endpoint *ep;
    int64_t n_ep, cap_ep;
    or_pending *stack;
    int64_t n_st, cap_st;
    uint64_t *tally; /* [L+1] */
    double *signal;  /* [signal_bins] induced charge per time bin (units of e) */
    int err;
} or_aval_out;

static int push_pending(or_aval_out *o, const or_pending *p)
{
    if (o->n_st == o->cap_st) {
        int64_t nc = o->cap_st ? 2 * o->cap_st : 64;
        or_pending *ns = (or_pending *)realloc(o->stack, sizeof(or_pending) * nc);
        if (!ns) return -1;
        o->stack = ns;
        o->cap_st = nc;
    }
    o->stack[o->n_st++] = *p;
    return 0;
}

static or_endpoint *new_endpoint(or_aval_out *o)
{
    if (o->n_ep == o->cap_ep) {
        int64_t nc = o->cap_ep ? 2 * o->cap_ep : 64;
        or_endpoint *ne = (or_endpoint *)realloc(o->ep, sizeof(or_endpoint) * nc);
        if (!ne) return NULL;
        o->ep = ne;
        o->cap_ep = nc;
    }
    or_endpoint *e = &o->ep[o->n_ep++];
    memset(e, 0, sizeof(*e));
    return e;
}

static double kinetic_energy(const double v[3]) { return dot3(v, v) / (2.0 * OR_ACCEL_PER_VCM); }
static double speed_of(double eps) { return sqrt(2.0 * OR_ACCEL_PER_VCM * eps); }

static void isotropic(double u_cos, double u_phi, double n[3])
{
    double ct = 1.0 - 2.0 * u_cos;
    double st2 = 1.0 - ct * ct;
    double st = st2 > 0.0 ? sqrt(st2) : 0.0;
    double phi = 2.0 * OR_PI * u_phi;
    n[0] = st * cos(phi);
    n[1] = st * sin(phi);
    n[2] = ct;
}

/* Anisotropy of level j at energy eps: the constant xi0 when the level's
 * screening energy is 0, else eps / (eps + screen) (the screened-Coulomb
 * form, forward-peaked at high energy). */
static double level_xi(const or_table *t, int j, double eps)
{
    if (t->screen[j] > 0.0) return eps / (eps + t->screen[j]);
    return t->xi0[j];
}

/* New unit direction of a scattered electron with incident velocity v.
 * xi = 0: isotropic in the lab frame (cos theta = 1 - 2 u_cos, phi = 2 pi
 * u_phi).  Otherwise the deflection chi from the incident direction has the
 * screened-Coulomb density p(mu) = (1 - xi^2) / (2 (1 - xi mu)^2) in
 * mu = cos chi (Okhrimovskyy, Bogaerts, Gijbels, Phys. Rev. E 65, 037402,
 * 2002), sampled by inverting its distribution function:
 *   mu = (1 + xi - 2 u_cos) / (1 + xi - 2 xi u_cos),
 * and the azimuth 2 pi u_phi turns about the incident direction d in the
 * orthonormal frame (e1, e2, d) of Duff et al., "Building an orthonormal
 * basis, revisited", JCGT 6(1), 2017.  A resting electron has d = +z.
 * Returns mu (cos chi; for xi = 0 the lab cos theta). */
static double scatter(double xi, const double v[3], double u_cos, double u_phi, double n[3])
{
    if (xi == 0.0) {
        isotropic(u_cos, u_phi, n);
        double sp = sqrt(dot3(v, v));
        return sp > 0.0 ? dot3(v, n) / sp : n[2];
    }
    double den = 1.0 + xi - 2.0 * xi * u_cos;
    double mu = (1.0 + xi - 2.0 * u_cos) / den;
    double one_minus = 2.0 * u_cos * (1.0 - xi) / den; /* 1 - mu without cancellation */
    double s2 = one_minus * (2.0 - one_minus);
    double sc = s2 > 0.0 ? sqrt(s2) : 0.0;               /* sin chi */
    double sp = sqrt(dot3(v, v));
    double d[3] = {0.0, 0.0, 1.0};
    if (sp > 0.0) {
        d[0] = v[0] / sp; d[1] = v[1] / sp; d[2] = v[2] / sp;
    }
    double sg = d[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + d[2]);
    double b = d[0] * d[1] * a;
    double e1[3] = {1.0 + sg * d[0] * d[0] * a, sg * b, -sg * d[0]};
    double e2[3] = {b, sg + d[1] * d[1] * a, -d[1]};
    double phi = 2.0 * OR_PI * u_phi;
    double c = cos(phi), s = sin(phi);
    for (int k = 0; k < 3; ++k) n[k] = mu * d[k] + sc * (c * e1[k] + s * e2[k]);
    return mu;
}

/* Test hook: scatter() above. */
double or_scatter(double xi, const double v[3], double u_cos, double u_phi, double n[3])
{
    return scatter(xi, v, u_cos, u_phi, n);
}

/* Elastic collision on a heavy target at rest: new direction n from
 * scatter(); the energy is scaled by 1 - recoil*(1 - cos chi), chi the lab
 * deflection angle and recoil = 2m/M (first order in m/M of the two-body
 * kinematics).  Writes the new velocity. */
void or_elastic(double recoil, double xi, const double v[3], double u_cos, double u_phi,
                double v_out[3])
{
    double n[3];
    double eps = kinetic_energy(v);
    double sp = sqrt(dot3(v, v));
    scatter(xi, v, u_cos, u_phi, n);
    double cchi = sp > 0.0 ? dot3(v, n) / sp : 0.0;
    double s = speed_of(eps * (1.0 - recoil * (1.0 - cchi)));
    v_out[0] = s * n[0]; v_out[1] = s * n[1]; v_out[2] = s * n[2];
}

/* Energy of the new electron of an ionisation from the remainder
 * rest = eps - I: uniform on [0, rest] (w = 0), or with density
 * proportional to 1 / (1 + (x / w)^2) on [0, rest / 2] (the form of Opal,
 * Peterson and Beaty, J. Chem. Phys. 55, 4100, 1971), by inversion
 * x = w tan(u atan(rest / (2 w))). */
static double ionisation_share(double w, double rest, double u)
{
    if (w <= 0.0) return u * rest;
    return w * tan(u * atan(rest / (2.0 * w)));
}

/* Test hook: ionisation_share() above. */
double or_ionisation_share(double w, double rest, double u) { return ionisation_share(w, rest, u); }

/* Transport one electron until its status is non-zero (Fig. 2, dashed box). */
static void transport_electron(const or_table *tb, const or_field *f, const or_run_args *a,
                               int32_t aval, double plate_e, const or_pending *start,
                               or_aval_out *o)
{
    double r[3] = {start->r[0], start->r[1], start->r[2]};
    double v[3] = {start->v[0], start->v[1], start->v[2]};
    double t = start->t;
    uint32_t n_flight = 0, n_real = 0;
    double work = 0.0, inel = 0.0, recoil = 0.0, share = 0.0;
    double w[3] = {-OR_OMEGA_PER_T * f->b[0], -OR_OMEGA_PER_T * f->b[1],
                   -OR_OMEGA_PER_T * f->b[2]}; /* electron: q = -e */
    const int has_b = f->b[0] != 0.0 || f->b[1] != 0.0 || f->b[2] != 0.0;
    const int signal = a->signal_kind != OR_W_NONE && a->signal_bins > 0;
    or_signal sg;
    if (signal) signal_start(a, f, &sg, t, r);
    int status = or_boundary(f, r);
    while (status == 0) {
        if (n_flight == 0xFFFFFFFFu) {
            status = OR_FLIGHT_LIMIT;
            break;
        }
        const uint32_t flight = n_flight;
        double u[4];
        draw4(a->seed, aval + a->aval_base, start->uid, flight, 0u, u);
        /* field at the start of the flight, held for the flight */
        double E[3];
        or_field_eval(f, plate_e, r, E);
        double acc[3] = {-OR_ACCEL_PER_VCM * E[0], -OR_ACCEL_PER_VCM * E[1],
                         -OR_ACCEL_PER_VCM * E[2]};
        /* null-collision free flight.  With the banded majorant a flight
         * longer than the window tau stops at tau without a collision test
         * (memoryless restart). */
        double nu = tb->nu_max;
        double dt;
        int pseudo = 0;
        if (a->majorant == 1) {
            double tau;
            nu = banded_majorant(tb, v, E, has_b, a->window, &tau);
            dt = -log(u[0]) / nu;
            if (dt >= tau) {
                dt = tau;
                pseudo = 1;
            }
        } else {
            dt = -log(u[0]) / nu;
        }
        int timed = 0;
        if (a->t_max > 0.0 && t + dt > a->t_max) {
            dt = a->t_max - t;
            timed = 1;
        }
        /* The flight, in `ns` equal sub-steps with the field evaluated at
         * the start of each (ns = 1: the field of the flight's start is
         * held).  With `crossing`, a sub-step that leaves the volume ends at
         * its first boundary crossing. */
        const int ns = a->substeps > 1 ? a->substeps : 1;
        const double h = ns > 1 ? dt / ns : dt;
        double t_end = timed ? a->t_max : t + dt;
        for (int sub = 0; sub < ns; ++sub) {
            if (sub > 0) {
                or_field_eval(f, plate_e, r, E);
                for (int d = 0; d < 3; ++d) acc[d] = -OR_ACCEL_PER_VCM * E[d];
            }
            double r0[3] = {r[0], r[1], r[2]}, v0[3] = {v[0], v[1], v[2]};
            or_flight(r, v, acc, w, h);
            status = or_boundary(f, r);
            double tc = h;
            if (a->crossing && f->kind == OR_PLATE && !has_b) {
                /* the vertex comes before the end: if it is outside, the
                 * first crossing lies before it */
                int sv = plate_vertex_exit(f, r0, v0, acc, h, &tc);
                if (sv) status = sv;
            }
            double te = sub == ns - 1 ? t_end : t + (sub + 1) * h; /* this step's end */
            if (a->crossing && status) {
                double hs = first_exit(f, r0, v0, acc, w, tc);
                r[0] = r0[0]; r[1] = r0[1]; r[2] = r0[2];
                v[0] = v0[0]; v[1] = v0[1]; v[2] = v0[2];
                or_flight(r, v, acc, w, hs);
                status = or_boundary(f, r);
                t_end = te = t + sub * h + hs;
            } else if (status && sub < ns - 1) {
                t_end = te;
            }
            if (signal) signal_step(a, f, &sg, o->signal, r0, v0, acc, w, t + sub * h, te);
            /* work done by the field on the electron (eV): -E . dr */
            work += -(E[0] * (r[0] - r0[0]) + E[1] * (r[1] - r0[1]) + E[2] * (r[2] - r0[2]));
            if (status) break;
        }
        t = t_end;
        n_flight = flight + 1u;
        if (status) break;
        if (timed) {
            status = OR_TIME;
            break;
        }
        if (pseudo) continue; /* window ended before a collision */
        double eps = kinetic_energy(v);
        int lvl = table_select(tb, eps, u[1], nu);
        if (lvl < 0) {
            o->tally[tb->L] += 1;
            continue;
        }
        o->tally[lvl] += 1;
        if (tb->type[lvl] == OR_ATTACHMENT) { /* captured: the electron ends here */
            status = OR_ATTACHED;
            break;
        }
        const double xi = level_xi(tb, lvl, eps);
        if (tb->type[lvl] == OR_ELASTIC) {
            or_elastic(tb->recoil, xi, v, u[2], u[3], v);
            recoil += eps - kinetic_energy(v);
        } else {
            double n[3];
            scatter(xi, v, u[2], u[3], n);
            double eps_new = eps - tb->thr[lvl];
            inel += tb->thr[lvl];
            if (tb->type[lvl] == OR_IONISATION) {
                /* the remainder is shared (ionisation_share); the new
                 * electron starts here, now, in an independent isotropic
                 * direction */
                double u2[4];
                draw4(a->seed, aval + a->aval_base, start->uid, flight, 1u, u2);
                double eps_sec = ionisation_share(tb->split_w, eps_new, u2[0]);
                eps_new = eps_new - eps_sec;
                share += eps_sec;
                double ns[3];
                isotropic(u2[1], u2[2], ns);
                double s = speed_of(eps_sec);
                or_pending child;
                child.r[0] = r[0]; child.r[1] = r[1]; child.r[2] = r[2];
                child.t = t;
                child.e0 = eps_sec;
                child.v[0] = s * ns[0]; child.v[1] = s * ns[1]; child.v[2] = s * ns[2];
                child.uid = or_child_uid(start->uid, flight);
                if (push_pending(o, &child)) {
                    o->err = -1;
                    return;
                }
            }
            double s = speed_of(eps_new);
            v[0] = s * n[0]; v[1] = s * n[1]; v[2] = s * n[2];
        }
        n_real += 1u;
        if (a->coll_limit && n_real >= a->coll_limit) {
            status = OR_COLL_LIMIT;
            break;
        }
    }
    if (signal) signal_end(a, f, &sg, o->signal, r);
    or_endpoint *e = new_endpoint(o);
    if (!e) {
        o->err = -1;
        return;
    }
    e->x0 = start->r[0]; e->y0 = start->r[1]; e->z0 = start->r[2];
    e->t0 = start->t; e->e0 = start->e0;
    e->x1 = r[0]; e->y1 = r[1]; e->z1 = r[2];
    e->t1 = t; e->e1 = kinetic_energy(v);
    e->status = status;
    e->n_flight = n_flight;
    e->uid = start->uid;
    e->ledger[0] = work; e->ledger[1] = inel; e->ledger[2] = recoil; e->ledger[3] = share;
}

/* ------------------------------------------------ driver */
typedef struct {
    const or_table *tb;
    const or_field *f;
    const or_run_args *a;
    const int64_t *first;  /* [n_aval+1] offsets into order[] */
    const int64_t *order;  /* primaries sorted by avalanche, stable */
    or_aval_out *out;      /* [n_aval] */
    int32_t next;          /* shared work counter */
    pthread_mutex_t lock;
} or_job;

static void run_avalanche(or_job *J, int32_t av)
{
    or_aval_out *o = &J->out[av];
    const or_run_args *a = J->a;
    double plate_e = a->aval_field ? a->aval_field[av] : J->f->e0;
    o->tally = (uint64_t *)calloc((size_t)J->tb->L + 1, sizeof(uint64_t));
    o->signal = (double *)calloc((size_t)(a->signal_bins > 0 ? a->signal_bins : 1), sizeof(double));
    if (!o->tally || !o->signal) {
        o->err = -1;
        return;
    }
    /* Push the primaries in reverse so they are taken in input order. */
    for (int64_t q = J->first[av + 1] - 1; q >= J->first[av]; --q) {
        int64_t p = J->order[q];
        double s = speed_of(a->e[p]);
        or_pending e;
        e.r[0] = a->x[p]; e.r[1] = a->y[p]; e.r[2] = a->z[p];
        e.t = a->t[p];
        e.e0 = a->e[p];
        e.v[0] = s * a->dx[p]; e.v[1] = s * a->dy[p]; e.v[2] = s * a->dz[p];
        e.uid = a->uid[p];
        if (push_pending(o, &e)) {
            o->err = -1;
            return;
        }
    }
    /* "Next electron" until the stack is empty (Fig. 2). */
    while (o->n_st > 0 && !o->err) {
        or_pending e = o->stack[--o->n_st];
        transport_electron(J->tb, J->f, a, av, plate_e, &e, o);
    }
}

static void *worker(void *arg)
{
    or_job *J = (or_job *)arg;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int32_t av = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (av >= J->a->n_avalanches) break;
        run_avalanche(J, av);
    }
    return NULL;
}

typedef struct {
    int32_t n_aval, L;
    or_aval_out *out;
    int64_t total;
} or_result;

/* Run every avalanche.  Returns 0 and a result handle, or a negative code:
 * -1 out of memory, -2 bad gas table, -3 bad arguments. */
int or_run(const or_gas *g, const or_field *f, const or_run_args *a, or_result **res)
{
    *res = NULL;
    if (a->n_avalanches < 0 || a->n_primaries < 0) return -3;
    if (f->kind == OR_GRID && (f->nx < 2 || f->ny < 2 || f->nz < 2 || !f->grid)) return -3;
    if (f->kind == OR_MESH) {
        if (f->n_tets < 1 || f->n_mesh_nodes < 4 || !f->mesh_nodes || !f->mesh_tets ||
            !f->mesh_values)
            return -3;
        for (int64_t i = 0; i < 4 * f->n_tets; ++i)
            if (f->mesh_tets[i] < 0 || f->mesh_tets[i] >= f->n_mesh_nodes) return -3;
    }
    for (int64_t p = 0; p < a->n_primaries; ++p)
        if (a->aval[p] < 0 || a->aval[p] >= a->n_avalanches) return -3;
    if (a->substeps < 0 || a->crossing < 0 || a->crossing > 1) return -3;
    if (a->signal_kind < OR_W_NONE || a->signal_kind > OR_W_MAP) return -3;
    if (a->signal_kind != OR_W_NONE &&
        (a->signal_bins < 0 || !(a->signal_dt > 0.0) || !isfinite(a->signal_t0) ||
         (a->signal_kind == OR_W_PLATE && f->kind != OR_PLATE) ||
         (a->signal_kind == OR_W_COAX && f->kind != OR_COAX && f->kind != OR_GRID &&
          f->kind != OR_MESH) ||
         (a->signal_kind == OR_W_MAP && f->kind != OR_GRID && f->kind != OR_MESH)))
        return -3;
    or_table tb;
    if (table_build(g, &tb)) return -2;
    tb.field_emax = a->substeps > 1 ? field_emax(f) : 0.0;
    if (a->majorant == 1) {
        if (!(a->window > 0.0) || !(a->band_width > 0.0) || bands_build(&tb, a->band_width)) {
            free(tb.cum);
            return -3;
        }
    }
    int32_t A = a->n_avalanches;
    int64_t *first = (int64_t *)calloc((size_t)A + 1, sizeof(int64_t));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(a->n_primaries + 1));
    or_aval_out *out = (or_aval_out *)calloc((size_t)A + 1, sizeof(or_aval_out));
    if (!first || !order || !out) {
        free(first); free(order); free(out); free(tb.cum); free(tb.bmax);
        return -1;
    }
    for (int64_t p = 0; p < a->n_primaries; ++p) first[a->aval[p] + 1] += 1;
    for (int32_t k = 0; k < A; ++k) first[k + 1] += first[k];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)A + 1));
        if (!fill) {
            free(first); free(order); free(out); free(tb.cum); free(tb.bmax);
            return -1;
        }
        memcpy(fill, first, sizeof(int64_t) * ((size_t)A + 1));
        for (int64_t p = 0; p < a->n_primaries; ++p) order[fill[a->aval[p]]++] = p;
        free(fill);
    }
    or_job J;
    J.tb = &tb; J.f = f; J.a = a; J.first = first; J.order = order; J.out = out;
    J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    int nt = a->n_threads > 0 ? a->n_threads : 1;
    if (nt > 256) nt = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 0; i < nt; ++i)
        if (pthread_create(&th[i], NULL, worker, &J) == 0) ++started;
    if (started == 0) worker(&J);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&J.lock);
    free(first);
    free(order);
    int err = 0;
    int64_t total = 0;
    for (int32_t k = 0; k < A; ++k) {
        if (out[k].err) err = -1;
        total += out[k].n_ep;
        free(out[k].stack);
        out[k].stack = NULL;
    }
    or_result *R = (or_result *)malloc(sizeof(or_result));
    if (err || !R) {
        for (int32_t k = 0; k < A; ++k) {
            free(out[k].ep);
            free(out[k].tally);
        }
        free(out); free(R); free(tb.cum); free(tb.bmax);
        return -1;
    }
    R->n_aval = A;
    R->L = tb.L;
    R->out = out;
    R->total = total;
    free(tb.cum);
    free(tb.bmax);
    *res = R;
    return 0;
}

int64_t or_result_count(const or_result *R) { return R ? R->total : -1; }

/* Copy the endpoints (avalanche by avalanche, in stack order), the number
 * of electrons of each avalanche and its collision tallies ([L] real per
 * level, then null flights) into caller arrays.  ledger may be NULL. */
int or_result_fetch(const or_result *R, double *x0, double *y0, double *z0, double *t0,
                    double *e0, double *x1, double *y1, double *z1, double *t1, double *e1,
                    int32_t *status, int32_t *aval, uint64_t *uid, uint32_t *n_flight,
                    double *ledger, uint64_t *electrons, uint64_t *tallies)
{
    if (!R) return -3;
    int64_t i = 0;
    for (int32_t k = 0; k < R->n_aval; ++k) {
        const or_aval_out *o = &R->out[k];
        electrons[k] = (uint64_t)o->n_ep;
        for (int j = 0; j <= R->L; ++j) tallies[(int64_t)k * (R->L + 1) + j] = o->tally[j];
        for (int64_t q = 0; q < o->n_ep; ++q, ++i) {
            const or_endpoint *e = &o->ep[q];
            x0[i] = e->x0; y0[i] = e->y0; z0[i] = e->z0; t0[i] = e->t0; e0[i] = e->e0;
            x1[i] = e->x1; y1[i] = e->y1; z1[i] = e->z1; t1[i] = e->t1; e1[i] = e->e1;
            status[i] = e->status;
            aval[i] = k;
            uid[i] = e->uid;
            n_flight[i] = e->n_flight;
            if (ledger)
                for (int m = 0; m < 4; ++m) ledger[4 * i + m] = e->ledger[m];
        }
    }
    return 0;
}

/* Per-avalanche signals, [n_aval][bins]. */
int or_result_signal(const or_result *R, int32_t bins, double *out)
{
    if (!R || bins < 0) return -3;
    for (int32_t k = 0; k < R->n_aval; ++k)
        for (int32_t j = 0; j < bins; ++j) out[(int64_t)k * bins + j] = R->out[k].signal[j];
    return 0;
}

void or_result_free(or_result *R)
{
    if (!R) return;
    for (int32_t k = 0; k < R->n_aval; ++k) {
        free(R->out[k].ep);
        free(R->out[k].tally);
        free(R->out[k].signal);
    }
    free(R->out);
    free(R);
}

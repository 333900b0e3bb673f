// gt_device.cuh -- device-side state and the per-flight step of the
// microscopic avalanche transport (arXiv:2509.15377, Sec. 2, Fig. 2), for
// sm_103a.  Two precisions share the structure of the step:
//   Fp64Electron   every quantity in FP64;
//   MixedElectron  FP32 kinematics, field, table interpolation and
//                  scattering; FP64 absolute position and time (FP32 offsets
//                  since the last flush are folded into FP64 every round),
//                  and FP64 decisions for the level-threshold and boundary
//                  tests (an FP32 pre-test with a margin, confirmed in FP64
//                  only inside the margin, takes the FP64 decision exactly).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gt_avalanche.h"

namespace gt {

// ---------------------------------------------------------------- units
// e/m = 1.75882001076e11 C/kg (CODATA 2018): acceleration per V/cm in
// cm/ns^2 and cyclotron rate per T in rad/ns.
constexpr double kAccel = 1.75882001076e-3;
constexpr double kOmega = 175.882001076;
constexpr double kTwoAccel = 2.0 * kAccel;          // v^2 = kTwoAccel * eps
constexpr double kInvTwoAccel = 1.0 / kTwoAccel;    // eps = v^2 * kInvTwoAccel
constexpr double kTwoPi = 6.283185307179586476925;
constexpr float kAccelF = 1.75882001076e-3f;
constexpr float kTwoAccelF = (float)(2.0 * 1.75882001076e-3);
constexpr float kInvTwoAccelF = (float)(1.0 / (2.0 * 1.75882001076e-3));
constexpr float kTwoPiF = 6.28318530717958647692f;

enum : int { EV_NONE = 0, EV_CHILD = 1, EV_RETIRE = 2 };

// ------------------------------------------------------------ parameters
struct DevGas {
    int n_levels, n_nodes;
    double d_eps, inv_d_eps, nu_max, inv_nu_max, recoil;
    float inv_d_eps_f, nu_max_f, inv_nu_max_f, recoil_f;
    float last_x_f, lastk_f;  // n_nodes - 1 and n_nodes - 2 as floats
    const double *cum64;  // [n_nodes][n_levels] running sums over levels
    const float *cum32;
    // Banded majorant: band b covers nodes [b n, (b+1) n]; bandmax tables
    // hold range maxima, level j, entry b = max over bands b .. b + 2^j - 1
    // (a sparse table: the maximum over any band range is two lookups).
    int n_bands, band_levels;
    int bands_monotone;          // band bounds non-decreasing: the range maximum is the top band's
    int level0_elastic;          // level 0 is an elastic level
    double inv_band_width;       // 1 / (n d_eps)
    float inv_band_width_f, last_band_f;
    const double *band64;        // [band_levels][n_bands]
    const float *band32;
    int32_t type[GT_MAX_LEVELS];
    double thr[GT_MAX_LEVELS];
    // angular model per level (xi0 where screen == 0, else eps/(eps+screen))
    // and the ionisation sharing width; any_aniso = 0 when all isotropic
    double xi0[GT_MAX_LEVELS], screen[GT_MAX_LEVELS];
    double split_w;
    float split_w_f;
    int any_aniso;
    int any_special;  // anisotropy, attachment or a sharing law (general step)
};

struct DevField {
    int kind;
    int has_b;
    double e0, gap;
    double wire_r2, tube_r2, coax_k;   // coax_k = V / ln(b/a)
    double w[3];                       // magnetic rotation vector -kOmega*B
    int nx, ny, nz;
    double origin[3], inv_spacing[3], hi[3];
    const float4 *grid;
    // FP32 copies for the mixed-precision step (no per-flight conversions)
    float e0_f, coax_k_f, w_f[3];
    float origin_f[3], inv_spacing_f[3];
    float wire_r2_hi_f, tube_r2_lo_f;    // radial pre-test limits (1e-5 margins)
    float box_lo_f[3], box_hi_f[3];      // map-box pre-test limits (inside by 1e-5)
    float cell_hi_f[3], node_hi_f[3];    // n - 2 and n - 1 per axis
    double emax;                         // largest |E| of the volume (COAX, GRID; else 0)
    double inv_gap;                      // PLATE: 1 / gap (anode weighting potential)
    double ln_tube, inv_ln_ab;           // COAX/GRID wire: ln b, 1 / ln(a/b)
    // MESH: element records (kMeshRec values each, FP32 and FP64) and the
    // uniform bins of the element search over the mesh's box (origin..hi)
    const float4 *tet32;
    const double *tet64;
    const int4 *tet_nb;                  // element across the face opposite node i (-1: none)
    const int *bin_start;                // [bins + 1] offsets into bin_tets
    const int *bin_tets;                 // elements meeting each bin, ascending
    int bin_n[3];
    double bin_lo[3], bin_inv[3];        // box corner, bins per cm
    float bin_lo_f[3], bin_inv_f[3];
};

struct Header {  // at the start of the work space, 256 bytes
    unsigned long long head;      // next queue ticket
    unsigned long long tail;      // slots reserved (stored or dropped)
    unsigned long long done;      // electrons finished or dropped
    unsigned long long dropped;   // secondaries not stored
    unsigned long long flights, real, nul;
    unsigned int error;           // ERR_* bits
    unsigned int pad0;
    unsigned long long n_new[2];  // plain mode: secondaries of this generation
    unsigned long long n_next[2]; // plain mode: electrons of next generation
    unsigned long long t_start;   // %globaltimer at the start of the run
    unsigned long long pad[19];
};
static_assert(sizeof(Header) == 256, "header size");

constexpr unsigned ERR_OVERFLOW = 1u, ERR_TIMEOUT = 2u, ERR_BADARG = 4u;

// Electron state parked between generations (plain mode), SoA.
struct Stack {
    double *x, *y, *z, *t, *vx, *vy, *vz;
    uint32_t *nf, *nreal;
    uint64_t *uid;
    int64_t *slot;
    int32_t *alive;
};

struct RunParams {
    DevGas gas;
    DevField field;
    // endpoint arrays (caller)
    double *x0, *y0, *z0, *t0, *e0, *x1, *y1, *z1, *t1, *e1;
    int32_t *status, *aval;
    uint64_t *uid;
    uint32_t *nflight;
    uint64_t *tallies;    // [n_avalanches][n_levels + 1]
    uint64_t *electrons;  // [n_avalanches]
    int64_t capacity;
    // work space
    Header *hdr;
    unsigned int *ready;      // [capacity] queue slot filled
    double *bvx, *bvy, *bvz;  // [capacity] velocity at birth
    int32_t *belem;           // [capacity] MESH: element of the birth point (-1: unknown)
    unsigned long long *created;  // [n_avalanches] (size_limit only)
    const double *aval_field;     // [n_avalanches] or null
    // run options
    uint64_t seed;
    double t_max;
    uint32_t coll_limit;
    int refill_period;  // batched: collision rounds between queue refills
    int flights_per_phase;  // batched mixed: flights before a warp's collisions
    int majorant;           // GT_MAJORANT_GLOBAL / GT_MAJORANT_BANDED
    double window;          // banded: window factor c
    float window_f;
    int substeps;           // field evaluations per flight (1: held field)
    int crossing;           // 1: leaving electrons end at the first crossing
    int signal_kind;        // readout electrode (GT_W_*), GT_W_NONE: no signal
    int signal_bins;
    double signal_t0, signal_dt, signal_inv_dt;
    double *signal;         // [n_avalanches][signal_bins]
    double field_emax;      // > 0: bound |E| by this in the banded majorant
    float field_emax_f;
    uint64_t size_limit;
    long long spin_limit_ns, time_limit_ns;
    int n_avalanches;
    int aval_base;          // workload number of avalanche 0 (random-stream counter only)
    uint32_t rk[20];        // Philox round keys of the seed: (k0, k1) of rounds 0..9
};

// --------------------------------------------------------- small helpers
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int lanemask_lt()
{
    unsigned int m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ------------------------------------------------------- random numbers
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (c0,c1,c2,c3) -> (hi(B*c2)^c1^k0, lo(B*c2), hi(A*c0)^c3^k1, lo(A*c0)),
// A = 0xD2511F53, B = 0xCD9E8D57, with the key bumped by (0x9E3779B9,
// 0xBB67AE85) after each round.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo_a = 0xD2511F53u * c.x, hi_a = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo_b = 0xCD9E8D57u * c.z, hi_b = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi_b ^ c.y ^ k0, lo_b, hi_a ^ c.w ^ k1, lo_a);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Stream of electron `uid` in avalanche `aval`: key (seed_lo, seed_hi),
// counter (flight, 2 aval + sub, uid_lo, uid_hi).
__device__ __forceinline__ uint4 draw(uint64_t seed, int aval, uint64_t uid, uint32_t flight,
                                      uint32_t sub)
{
    return philox10(make_uint4(flight, ((uint32_t)aval << 1) | sub, (uint32_t)uid,
                               (uint32_t)(uid >> 32)),
                    (uint32_t)seed, (uint32_t)(seed >> 32));
}

// The same with the round keys of the seed taken from the run parameters
// (rk[2r], rk[2r + 1] = key + r * Weyl constants): the key schedule costs no
// instruction per block.
__device__ __forceinline__ uint4 draw_rk(const uint32_t (&rk)[20], int aval, uint64_t uid,
                                         uint32_t flight, uint32_t sub)
{
    uint4 c = make_uint4(flight, ((uint32_t)aval << 1) | sub, (uint32_t)uid,
                         (uint32_t)(uid >> 32));
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo_a = 0xD2511F53u * c.x, hi_a = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo_b = 0xCD9E8D57u * c.z, hi_b = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi_b ^ c.y ^ rk[2 * r], lo_b, hi_a ^ c.w ^ rk[2 * r + 1], lo_a);
    }
    return c;
}

// (w + 1/2) 2^-32 in (0, 1), exact in FP64.
__device__ __forceinline__ double u01d(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }
// (w>>9 + 1/2) 2^-23 in (0, 1), exact in FP32 (24 significant bits).  Built
// from the bits (1 + (w>>9) 2^-23 has exponent 0) so that no int-to-float
// conversion is issued: conversions share GB300's narrow FP64 pipe.
__device__ __forceinline__ float u01f(uint32_t w)
{
    return __uint_as_float(0x3F800000u | (w >> 9)) - (1.0f - 0x1p-24f);
}

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014); the id of
// the electron created in flight `flight` of `parent`.
__device__ __forceinline__ uint64_t child_uid(uint64_t parent, uint32_t flight)
{
    uint64_t z = parent + 0x9E3779B97F4A7C15ull * ((uint64_t)flight + 1ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ------------------------------------------------------- shared tables
// Per-CTA view of the gas constants; the FP32 cumulative table is staged
// into shared memory when it fits (mixed precision).
struct Tables {
    const float *band32;    // shared: banded-majorant range maxima (FP32)
    const float *cum32;     // shared or global, rows of `stride32` floats
    const double *cum64;    // global (read-only path), rows of n_levels
    const int *type;        // shared [L]
    const double *thr;      // shared [L]
    const float *thr_f;     // shared [L]
    const float *xi0_f;     // shared [L]
    const float *screen_f;  // shared [L]
    uint32_t *tally;        // shared [L][blockDim]: real collisions per level
    double *base;           // shared [4][blockDim]: FP64 position/time bases (mixed)
    int stride32;           // odd in shared memory: rows start on every bank
};

// ------------------------------------------------------ tetrahedral mesh
// An element record (built by field_setup from the element's nodes), as
// eight rows of four values: the first node v0 (and, in the FP32 record, the
// element's margin: a bound on the FP32 error of its barycentric
// coordinates, with a factor 2 to spare); the rows of M, the inverse
// of the edge matrix [v1 - v0, v2 - v0, v3 - v0], so that the barycentric
// coordinates of r are l1..l3 = M (r - v0) and l0 = 1 - l1 - l2 - l3; the
// field and weighting potential at v0; and their gradients in the element
// (row c: dE_c/dx, dE_c/dy, dE_c/dz, dphi/dx_c), so that the linear
// interpolation of the nodal values is E(r) = E(v0) + G (r - v0).
constexpr int kMeshRec = 32;

// Smallest barycentric coordinate of r in the element record q, in units of
// the element's FP32 margin: >= 1 inside for sure, < -1 outside for sure.
__device__ __forceinline__ float tet_min32(const float4 *q, float x, float y, float z)
{
    const float4 v = __ldg(q), m0 = __ldg(q + 1), m1 = __ldg(q + 2), m2 = __ldg(q + 3);
    const float dx = x - v.x, dy = y - v.y, dz = z - v.z;
    const float l1 = fmaf(m0.x, dx, fmaf(m0.y, dy, m0.z * dz));
    const float l2 = fmaf(m1.x, dx, fmaf(m1.y, dy, m1.z * dz));
    const float l3 = fmaf(m2.x, dx, fmaf(m2.y, dy, m2.z * dz));
    return __fdividef(fminf(fminf(l1, l2), fminf(l3, 1.0f - l1 - l2 - l3)), v.w);
}

__device__ __forceinline__ double tet_min64(const double *q, double x, double y, double z)
{
    const double dx = x - q[0], dy = y - q[1], dz = z - q[2];
    const double l1 = q[4] * dx + q[5] * dy + q[6] * dz;
    const double l2 = q[8] * dx + q[9] * dy + q[10] * dz;
    const double l3 = q[12] * dx + q[13] * dy + q[14] * dz;
    return fmin(fmin(l1, l2), fmin(l3, 1.0 - l1 - l2 - l3));
}

// Bin of r (-1 when r is clearly outside the mesh's box; a point on the box
// or within rounding of it goes to the nearest bin).
template <typename R>
__device__ __forceinline__ int mesh_bin(const int n[3], const R lo[3], const R inv[3], R x, R y,
                                        R z)
{
    const R q[3] = {x, y, z};
    int c = 0;
#pragma unroll
    for (int d = 2; d >= 0; --d) {
        const R g = (q[d] - lo[d]) * inv[d];
        if (!(g > (R)(-1e-3)) || !(g < (R)n[d] + (R)(1e-3))) return -1;
        int k = (int)g;
        k = k < 0 ? 0 : (k >= n[d] ? n[d] - 1 : k);
        c = c * n[d] + k;
    }
    return c;
}

// Element search: the hint when it holds r with every barycentric
// coordinate >= tol (FP32: in units of the element's margin), else the
// first (lowest-index) element of r's bin that does; -1 if none.
__device__ __forceinline__ int mesh_find32(const DevField &f, float x, float y, float z, int hint,
                                           float tol)
{
    if (hint >= 0 && tet_min32(f.tet32 + (kMeshRec / 4) * (int64_t)hint, x, y, z) >= tol)
        return hint;
    const int c = mesh_bin<float>(f.bin_n, f.bin_lo_f, f.bin_inv_f, x, y, z);
    if (c < 0) return -1;
    const int e = __ldg(f.bin_start + c + 1);
    for (int i = __ldg(f.bin_start + c); i < e; ++i) {
        const int t = __ldg(f.bin_tets + i);
        if (tet_min32(f.tet32 + (kMeshRec / 4) * (int64_t)t, x, y, z) >= tol) return t;
    }
    return -1;
}

__device__ __forceinline__ int mesh_find64(const DevField &f, double x, double y, double z,
                                           int hint, double tol)
{
    if (hint >= 0 && tet_min64(f.tet64 + kMeshRec * (int64_t)hint, x, y, z) >= tol) return hint;
    const int c = mesh_bin<double>(f.bin_n, f.bin_lo, f.bin_inv, x, y, z);
    if (c < 0) return -1;
    const int e = f.bin_start[c + 1];
    for (int i = f.bin_start[c]; i < e; ++i) {
        const int t = f.bin_tets[i];
        if (tet_min64(f.tet64 + kMeshRec * (int64_t)t, x, y, z) >= tol) return t;
    }
    return -1;
}

// Walk from element t towards r (FP32): while r is not inside with every
// coordinate >= tol (margin units), step across the face opposite the node
// of the most negative coordinate; -1 when the walk leaves the mesh or takes
// more than kMeshWalk steps (the bins decide then).
constexpr int kMeshWalk = 8;

__device__ __forceinline__ int mesh_walk32(const DevField &f, float x, float y, float z, int t,
                                           float tol)
{
    for (int step = 0; step < kMeshWalk; ++step) {
        const float4 *q = f.tet32 + (kMeshRec / 4) * (int64_t)t;
        const float4 v = __ldg(q), m0 = __ldg(q + 1), m1 = __ldg(q + 2), m2 = __ldg(q + 3);
        const float dx = x - v.x, dy = y - v.y, dz = z - v.z;
        const float l1 = fmaf(m0.x, dx, fmaf(m0.y, dy, m0.z * dz));
        const float l2 = fmaf(m1.x, dx, fmaf(m1.y, dy, m1.z * dz));
        const float l3 = fmaf(m2.x, dx, fmaf(m2.y, dy, m2.z * dz));
        float mn = 1.0f - l1 - l2 - l3;
        int im = 0;
        if (l1 < mn) { mn = l1; im = 1; }
        if (l2 < mn) { mn = l2; im = 2; }
        if (l3 < mn) { mn = l3; im = 3; }
        if (mn >= tol * v.w) return t;
        const int4 nb = __ldg(f.tet_nb + t);
        t = im == 0 ? nb.x : im == 1 ? nb.y : im == 2 ? nb.z : nb.w;
        if (t < 0) return -1;
    }
    return -1;
}

// The FP64 search (closed elements) of the position r = (x, y, z), which is
// (x32, y32, z32) in FP32: an element is tested in FP64 only when its FP32
// test does not rule it out (every coordinate above minus its margin).
__device__ __forceinline__ int mesh_find_mixed(const DevField &f, double x, double y, double z,
                                               float x32, float y32, float z32, int hint)
{
    auto holds = [&](int t) {
        return tet_min32(f.tet32 + (kMeshRec / 4) * (int64_t)t, x32, y32, z32) >= -1.0f &&
               tet_min64(f.tet64 + kMeshRec * (int64_t)t, x, y, z) >= 0.0;
    };
    if (hint >= 0) {  // the hint, then its face neighbours
        if (holds(hint)) return hint;
        const int4 nb = __ldg(f.tet_nb + hint);
        if (nb.x >= 0 && holds(nb.x)) return nb.x;
        if (nb.y >= 0 && holds(nb.y)) return nb.y;
        if (nb.z >= 0 && holds(nb.z)) return nb.z;
        if (nb.w >= 0 && holds(nb.w)) return nb.w;
    }
    const int c = mesh_bin<double>(f.bin_n, f.bin_lo, f.bin_inv, x, y, z);
    if (c < 0) return -1;
    const int e = __ldg(f.bin_start + c + 1);
    for (int i = __ldg(f.bin_start + c); i < e; ++i) {
        const int t = __ldg(f.bin_tets + i);
        if (holds(t)) return t;
    }
    return -1;
}

// Field of element record q at r (linear interpolation of the nodal values).
__device__ __forceinline__ void mesh_field32(const float4 *q, float x, float y, float z, float &ex,
                                             float &ey, float &ez)
{
    const float4 v = __ldg(q), e = __ldg(q + 4), gx = __ldg(q + 5), gy = __ldg(q + 6),
                 gz = __ldg(q + 7);
    const float dx = x - v.x, dy = y - v.y, dz = z - v.z;
    ex = fmaf(gx.x, dx, fmaf(gx.y, dy, fmaf(gx.z, dz, e.x)));
    ey = fmaf(gy.x, dx, fmaf(gy.y, dy, fmaf(gy.z, dz, e.y)));
    ez = fmaf(gz.x, dx, fmaf(gz.y, dy, fmaf(gz.z, dz, e.z)));
}

// Field (c = 0..2) or weighting potential (c = 3) of FP64 element record q at r.
__device__ __forceinline__ double mesh_value64(const double *q, int c, double x, double y, double z)
{
    const double dx = x - q[0], dy = y - q[1], dz = z - q[2];
    if (c == 3) return q[19] + q[23] * dx + q[27] * dy + q[31] * dz;
    const double *g = q + 20 + 4 * c;
    return q[16 + c] + g[0] * dx + g[1] * dy + g[2] * dz;
}

// --------------------------------------------------------------- fields
template <int FK>
__device__ __forceinline__ void field64(const DevField &f, double plate_e, double x, double y,
                                        double z, double &ex, double &ey, double &ez)
{
    if (FK == GT_FIELD_UNIFORM) {
        ex = 0.0; ey = 0.0; ez = -f.e0;
    } else if (FK == GT_FIELD_PLATE) {
        ex = 0.0; ey = 0.0; ez = -plate_e;
    } else if (FK == GT_FIELD_COAX) {
        const double s = f.coax_k / (x * x + y * y);
        ex = s * x; ey = s * y; ez = 0.0;
    } else if (FK == GT_FIELD_MESH) {
        const int t = mesh_find64(f, x, y, z, -1, 0.0);
        if (t < 0) {
            ex = ey = ez = 0.0;
        } else {
            const double *q = f.tet64 + kMeshRec * (int64_t)t;
            ex = mesh_value64(q, 0, x, y, z);
            ey = mesh_value64(q, 1, x, y, z);
            ez = mesh_value64(q, 2, x, y, z);
        }
    } else {
        const double p[3] = {x, y, z};
        const int n[3] = {f.nx, f.ny, f.nz};
        int i[3];
        double w[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double g = (p[d] - f.origin[d]) * f.inv_spacing[d];
            int k = (int)floor(g);
            k = k < 0 ? 0 : (k > n[d] - 2 ? n[d] - 2 : k);
            i[d] = k;
            w[d] = g - k;
        }
        ex = ey = ez = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
            const double wt = (di ? w[0] : 1.0 - w[0]) * (dj ? w[1] : 1.0 - w[1]) *
                              (dk ? w[2] : 1.0 - w[2]);
            const float4 e = __ldg(f.grid + (((int64_t)(i[2] + dk) * f.ny + (i[1] + dj)) * f.nx +
                                             (i[0] + di)));
            ex += wt * (double)e.x; ey += wt * (double)e.y; ez += wt * (double)e.z;
        }
    }
}

template <int FK>
__device__ __forceinline__ void field32(const DevField &f, float plate_e, float x, float y, float z,
                                        float &ex, float &ey, float &ez)
{
    if (FK == GT_FIELD_UNIFORM) {
        ex = 0.f; ey = 0.f; ez = -f.e0_f;
    } else if (FK == GT_FIELD_PLATE) {
        ex = 0.f; ey = 0.f; ez = -plate_e;
    } else if (FK == GT_FIELD_COAX) {
        const float s = __fdividef(f.coax_k_f, x * x + y * y);
        ex = s * x; ey = s * y; ez = 0.f;
    } else if (FK == GT_FIELD_MESH) {
        const int t = mesh_find32(f, x, y, z, -1, -1.0f);
        if (t < 0) {
            ex = ey = ez = 0.f;
        } else {
            mesh_field32(f.tet32 + (kMeshRec / 4) * (int64_t)t, x, y, z, ex, ey, ez);
        }
    } else {
        // cell (clamped to the last one) and weights without int/float
        // conversions: floor(g) by a round-down add of 2^23
        float w3[3];
        int i3[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float g = fmaxf((d == 0 ? x : d == 1 ? y : z) - f.origin_f[d], 0.f) *
                            f.inv_spacing_f[d];
            const float t = __fadd_rd(fminf(g, f.cell_hi_f[d]), 8388608.0f);
            i3[d] = __float_as_int(t) - 0x4B000000;
            w3[d] = fminf(g, f.node_hi_f[d]) - (t - 8388608.0f);
        }
        const int ix = i3[0], iy = i3[1], iz = i3[2];
        const float wx = w3[0], wy = w3[1], wz = w3[2];
        const float4 *b = f.grid + (((int64_t)iz * f.ny + iy) * f.nx + ix);
        const int64_t sy = f.nx, sz = (int64_t)f.nx * f.ny;
        const float4 c000 = __ldg(b), c100 = __ldg(b + 1);
        const float4 c010 = __ldg(b + sy), c110 = __ldg(b + sy + 1);
        const float4 c001 = __ldg(b + sz), c101 = __ldg(b + sz + 1);
        const float4 c011 = __ldg(b + sz + sy), c111 = __ldg(b + sz + sy + 1);
        // interpolate along x, then y, then z: Ex and Ey together in paired
        // FP32 instructions (FFMA2, sm_100 and later: each half rounds as
        // fmaf), Ez alone; b - a as fma(a, -1, b), the same rounding as a
        // subtraction
        auto lerp = [](float a, float b, float t) { return fmaf(t, b - a, a); };
        auto lerp2 = [](float2 a, float2 b, float2 t) {
            return __ffma2_rn(t, __ffma2_rn(a, make_float2(-1.0f, -1.0f), b), a);
        };
        auto xy = [](const float4 &c) { return make_float2(c.x, c.y); };
        const float2 tx = make_float2(wx, wx), ty = make_float2(wy, wy), tz = make_float2(wz, wz);
        const float2 a00 = lerp2(xy(c000), xy(c100), tx), a10 = lerp2(xy(c010), xy(c110), tx);
        const float2 a01 = lerp2(xy(c001), xy(c101), tx), a11 = lerp2(xy(c011), xy(c111), tx);
        const float2 exy = lerp2(lerp2(a00, a10, ty), lerp2(a01, a11, ty), tz);
        const float z00 = lerp(c000.z, c100.z, wx), z10 = lerp(c010.z, c110.z, wx);
        const float z01 = lerp(c001.z, c101.z, wx), z11 = lerp(c011.z, c111.z, wx);
        ex = exy.x; ey = exy.y;
        ez = lerp(lerp(z00, z10, wy), lerp(z01, z11, wy), wz);
    }
}

// Boundary status of an FP64 position (0 inside).
template <int FK>
__device__ __forceinline__ int boundary64(const DevField &f, double x, double y, double z)
{
    if (FK == GT_FIELD_PLATE) {
        if (z >= f.gap) return GT_ST_ANODE;
        if (z < 0.0) return GT_ST_CATHODE;
    } else if (FK == GT_FIELD_COAX) {
        const double r2 = x * x + y * y;
        if (r2 <= f.wire_r2) return GT_ST_WIRE;
        if (r2 >= f.tube_r2) return GT_ST_TUBE;
    } else if (FK == GT_FIELD_GRID) {
        const double r2 = x * x + y * y;
        if (f.wire_r2 > 0.0 && r2 <= f.wire_r2) return GT_ST_WIRE;
        if (x < f.origin[0] || x > f.hi[0] || y < f.origin[1] || y > f.hi[1] ||
            z < f.origin[2] || z > f.hi[2])
            return GT_ST_OUT_OF_MAP;
    } else if (FK == GT_FIELD_MESH) {
        const double r2 = x * x + y * y;
        if (f.wire_r2 > 0.0 && r2 <= f.wire_r2) return GT_ST_WIRE;
        if (mesh_find64(f, x, y, z, -1, 0.0) < 0) return GT_ST_OUT_OF_MAP;
    }
    return 0;
}

// ---------------------------------------------------- flight kinematics
// Exact motion over dt with constant acceleration a and magnetic rotation
// vector w (dv/dt = a + v x w): the component along w-hat accelerates
// uniformly; across it the drift (a x w)/|w|^2 plus a rotation by -|w| dt.
template <typename R>
__device__ __forceinline__ void lorentz_step(const R w[3], R ax, R ay, R az, R dt, R &vx, R &vy,
                                             R &vz, R &dx, R &dy, R &dz)
{
    const R wn2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    const R wn = sqrt(wn2);
    const R bx = w[0] / wn, by = w[1] / wn, bz = w[2] / wn;
    const R vpar = vx * bx + vy * by + vz * bz;
    const R apar = ax * bx + ay * by + az * bz;
    const R gx = (ay * w[2] - az * w[1]) / wn2;  // (a x w)/|w|^2
    const R gy = (az * w[0] - ax * w[2]) / wn2;
    const R gz = (ax * w[1] - ay * w[0]) / wn2;
    const R ux = vx - vpar * bx - gx, uy = vy - vpar * by - gy, uz = vz - vpar * bz - gz;
    const R cx = by * uz - bz * uy, cy = bz * ux - bx * uz, cz = bx * uy - by * ux;  // b x u
    R s, c;
    sincos(wn * dt, &s, &c);
    const R sw = s / wn;
    const R cw = (R)(1) - c;
    const R cwn = cw / wn;
    const R par = vpar * dt + (R)(0.5) * apar * dt * dt;
    dx = par * bx + gx * dt + ux * sw - cx * cwn;
    dy = par * by + gy * dt + uy * sw - cy * cwn;
    dz = par * bz + gz * dt + uz * sw - cz * cwn;
    const R vp = vpar + apar * dt;
    vx = vp * bx + gx + ux * c - cx * s;
    vy = vp * by + gy + uy * c - cy * s;
    vz = vp * bz + gz + uz * c - cz * s;
}

// Cumulative-rate selection at energy eps for R = u1 * nu_max: the level j
// with cum_{j-1}(eps) <= R < cum_j(eps), or -1 for a null collision.
template <typename R, typename T>
__device__ __forceinline__ int select_level(const T *cum, int L, int N, R inv_d_eps, R eps, R Rv)
{
    R xk = eps * inv_d_eps;
    const R last = (R)(N - 1);
    if (xk > last) xk = last;
    int k = (int)xk;
    if (k > N - 2) k = N - 2;
    const R f = xk - (R)k;
    const T *c0 = cum + (int64_t)k * L;
    const T *c1 = c0 + L;
    const R top = (R)c0[L - 1] + f * ((R)c1[L - 1] - (R)c0[L - 1]);
    if (!(Rv < top)) return -1;
    int lvl = 0;
    for (int j = 0; j < L - 1; ++j) {
        const R cj = (R)c0[j] + f * ((R)c1[j] - (R)c0[j]);
        lvl += (cj <= Rv) ? 1 : 0;
    }
    return lvl;
}

// FP32 selection on a table with row stride `stride`, without int/float
// conversions: floor(x) for 0 <= x < 2^23 is the round-down sum x + 2^23
// read back as an integer.  Rows k and k+1 bracket the energy (the last
// interval extends to energies beyond the table).  The level is found by a
// branch-free binary search over the non-decreasing running sums.
__device__ __forceinline__ int select_level32(const float *cum, int stride, int L, float lastk,
                                              float last, float inv_d_eps, float eps, float Rv)
{
    const float xk = eps * inv_d_eps;
    const float t = __fadd_rd(fminf(xk, lastk), 8388608.0f);
    const int k = __float_as_int(t) - 0x4B000000;
    const float f = fminf(xk, last) - (t - 8388608.0f);
    const float *c0 = cum + k * stride;
    const float *c1 = c0 + stride;
    const float top = fmaf(f, c1[L - 1] - c0[L - 1], c0[L - 1]);
    if (!(Rv < top)) return -1;
    const int m = L - 1;  // levels below the last; the last is known to exceed R
    int pos = 0;
    if (m > 0) {
        for (int step = 1 << (31 - __clz(m)); step > 0; step >>= 1) {
            const int j = pos + step - 1;
            if (j < m && fmaf(f, c1[j] - c0[j], c0[j]) <= Rv) pos += step;
        }
    }
    return pos;
}

// Level of a real collision whose R = u1 nu is known to lie below the total
// rate at fraction f of the table interval starting at row c0 (stride
// `stride`): the first level whose running sum exceeds R, by a branch-free
// binary search over the levels below the last.
__device__ __forceinline__ int select_below_total32(const float *c0, int stride, int L, float f,
                                                    float Rv)
{
    const float *c1 = c0 + stride;
    const int m = L - 1;  // < GT_MAX_LEVELS = 32: at most five halvings
    int pos = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int j = pos + step - 1;
        if (j < m && fmaf(f, c1[j] - c0[j], c0[j]) <= Rv) pos += step;
    }
    return pos;
}

// ---------------------------------------------------- banded majorant
// Band of an energy: floor(eps / band width), clamped to the band range.
__device__ __forceinline__ int band_index64(const DevGas &g, double eps)
{
    const double x = eps * g.inv_band_width;
    if (!(x > 0.0)) return 0;
    if (x >= (double)g.n_bands) return g.n_bands - 1;
    const int b = (int)floor(x);
    return b < g.n_bands ? b : g.n_bands - 1;
}

__device__ __forceinline__ int band_index32(const DevGas &g, float eps)
{
    const float x = fminf(fmaxf(eps * g.inv_band_width_f, 0.0f), g.last_band_f);
    return __float_as_int(__fadd_rd(x, 8388608.0f)) - 0x4B000000;
}

// Largest rate over bands lo..hi from the sparse table (two lookups).
template <typename T>
__device__ __forceinline__ T band_range_max(const T *bt, int n_bands, int lo, int hi)
{
    const int j = 31 - __clz(hi - lo + 1);
    const T a = bt[j * n_bands + lo], b = bt[j * n_bands + hi - (1 << j) + 1];
    return a > b ? a : b;
}

// Energy range [lo, hi] of a flight within the window tau in the held field
// E.  Without B the flight is v + a t and the energy eps0 + g(t) with
// g(t) = -(v.E) t + (a1 |E|^2 / 2) t^2, a convex parabola: hi is its larger
// end, lo its vertex (t* = v.E / (a1 |E|^2) when inside the window) or its
// smaller end.  With B, |dv/dt| <= a1 |E| bounds the displacement, and the
// range is eps0 -+ |E| (|v| tau + a1 |E| tau^2 / 2).
__device__ __forceinline__ void reach64(int has_b, double emax, double eps0, double vx, double vy,
                                        double vz, double ex, double ey, double ez, double tau,
                                        double &lo, double &hi)
{
    if (emax > 0.0) {
        // a field re-evaluated along the flight: |dv/dt| <= a1 emax
        const double D = emax * (sqrt(vx * vx + vy * vy + vz * vz) * tau +
                                 0.5 * (kAccel * emax) * tau * tau);
        lo = eps0 - D;
        hi = eps0 + D;
    } else if (!has_b) {
        const double vE = vx * ex + vy * ey + vz * ez, E2 = ex * ex + ey * ey + ez * ez;
        const double gw = -vE * tau + 0.5 * kAccel * E2 * tau * tau;
        hi = eps0 + (gw > 0.0 ? gw : 0.0);
        if (vE <= 0.0) {
            lo = eps0;
        } else {
            const double ts = vE / (kAccel * E2);
            lo = ts < tau ? eps0 - 0.5 * vE * ts : eps0 + gw;
        }
    } else {
        const double Em = sqrt(ex * ex + ey * ey + ez * ez);
        const double D = Em * (sqrt(vx * vx + vy * vy + vz * vz) * tau +
                               0.5 * (kAccel * Em) * tau * tau);
        lo = eps0 - D;
        hi = eps0 + D;
    }
}

// FP32 version, widened by 1e-5 of the energies involved against rounding.
template <int FK>
__device__ __forceinline__ void reach32(int has_b, float emax, float eps0, float vx, float vy,
                                        float vz, float ex, float ey, float ez, float plate_e,
                                        float tau, float &lo, float &hi, bool need_lo = true)
{
    if (emax > 0.0f) {
        const float D = emax * fmaf(0.5f * kAccelF * emax * tau, tau,
                                    sqrtf(vx * vx + vy * vy + vz * vz) * tau) * 1.00001f;
        lo = eps0 - D;
        hi = eps0 + D;
    } else if (!has_b) {
        const float vE = FK == GT_FIELD_PLATE ? -vz * plate_e : fmaf(vx, ex, fmaf(vy, ey, vz * ez));
        const float E2 = FK == GT_FIELD_PLATE ? plate_e * plate_e
                                              : fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        const float q = 0.5f * kAccelF * E2 * tau * tau;  // the acceleration term of g(tau)
        const float gw = fmaf(-vE, tau, q);
        const float margin = 1e-5f * (eps0 + fabsf(vE) * tau + q);
        hi = eps0 + fmaxf(gw, 0.0f) + margin;
        float l = eps0;
        if (need_lo && vE > 0.0f) {
            const float ts = __fdividef(vE, kAccelF * E2);
            l = ts < tau ? fmaf(-0.5f * vE, ts, eps0) : eps0 + gw;
        }
        lo = l - margin;
    } else {
        const float Em = sqrtf(ex * ex + ey * ey + ez * ez);
        const float D = Em * fmaf(0.5f * kAccelF * Em * tau, tau,
                                  sqrtf(vx * vx + vy * vy + vz * vz) * tau) * 1.00001f;
        lo = eps0 - D;
        hi = eps0 + D;
    }
}

// Isotropic unit vector from two uniforms: cos(theta) = 1 - 2 u, phi = 2 pi v.
__device__ __forceinline__ void isotropic64(double u, double v, double &nx, double &ny,
                                            double &nz)
{
    const double ct = 1.0 - 2.0 * u;
    const double st2 = 1.0 - ct * ct;
    const double st = st2 > 0.0 ? sqrt(st2) : 0.0;
    double s, c;
    sincos(kTwoPi * v, &s, &c);
    nx = st * c; ny = st * s; nz = ct;
}

// Square root of q > 0 in FP32 from the hardware rsqrt and one Newton step
// in residual form: q (r + r h), h = 1/2 - q r^2 / 2 from an FMA.  Within
// about 2 ulp and without the bias that a refinement factor rounded near
// 1.0 has (float32 emulation over 1e7 arguments: mean relative error below
// 3e-11); 0 for q = 0.
__device__ __forceinline__ float sqrt_nr(float q)
{
    float r = rsqrtf(q);
    r = fmaf(r, fmaf(-0.5f * q * r, r, 0.5f), r);
    return q > 0.f ? q * r : 0.f;
}

// FP32 version.  The azimuth comes from the hardware sin/cos (no range
// reduction instructions); (c, s) is then rescaled to unit length with a
// Newton-refined rsqrt, so that |n| = 1 to rounding and the speed set from
// it carries no systematic error from collision to collision.
__device__ __forceinline__ void isotropic32(float u, float v, float &nx, float &ny, float &nz)
{
    const float ct = 1.0f - 2.0f * u;
    const float st = 2.0f * sqrt_nr(u * (1.0f - u));  // sqrt(1 - ct^2), well conditioned
    float s, c;
    __sincosf(kTwoPiF * v, &s, &c);
    const float g = fmaf(c, c, s * s);
    float r = rsqrtf(g);
    r = r * fmaf(-0.5f * g, r * r, 1.5f);
    const float sr = st * r;
    nx = sr * c; ny = sr * s; nz = ct;
}

// Anisotropy of level j at energy eps: xi0 where the screening energy is 0,
// else eps / (eps + screen) (screened-Coulomb form).
__device__ __forceinline__ double level_xi64(const DevGas &g, int j, double eps)
{
    return g.screen[j] > 0.0 ? eps / (eps + g.screen[j]) : g.xi0[j];
}

// New unit direction after a collision with anisotropy xi != 0: deflection
// chi from the incident velocity v with the screened-Coulomb density
// (1 - xi^2) / (2 (1 - xi mu)^2) in mu = cos chi, sampled by inversion,
// mu = (1 + xi - 2u) / (1 + xi - 2 xi u) (1 - mu = 2u (1 - xi) / (same),
// without cancellation); azimuth 2 pi w about the incident direction d in
// the orthonormal frame (e1, e2, d) of Duff et al., JCGT 6(1), 2017; a
// resting electron takes d = +z.  Returns mu.
__device__ __forceinline__ double scatter64(double xi, double vx, double vy, double vz, double u,
                                            double w, double &nx, double &ny, double &nz)
{
    const double den = 1.0 + xi - 2.0 * xi * u;
    const double mu = (1.0 + xi - 2.0 * u) / den;
    const double om = 2.0 * u * (1.0 - xi) / den;
    const double s2 = om * (2.0 - om);
    const double sc = s2 > 0.0 ? sqrt(s2) : 0.0;
    const double sp = sqrt(vx * vx + vy * vy + vz * vz);
    double d0 = 0.0, d1 = 0.0, d2 = 1.0;
    if (sp > 0.0) {
        d0 = vx / sp; d1 = vy / sp; d2 = vz / sp;
    }
    const double sg = d2 >= 0.0 ? 1.0 : -1.0;
    const double a = -1.0 / (sg + d2);
    const double b = d0 * d1 * a;
    double sn, cs;
    sincos(kTwoPi * w, &sn, &cs);
    nx = mu * d0 + sc * (cs * (1.0 + sg * d0 * d0 * a) + sn * b);
    ny = mu * d1 + sc * (cs * (sg * b) + sn * (sg + d1 * d1 * a));
    nz = mu * d2 + sc * (cs * (-sg * d0) + sn * (-d1));
    return mu;
}

// FP32 version; the direction is rescaled to unit length with a
// Newton-refined rsqrt so that the speed set from it carries no systematic
// error from collision to collision.
__device__ __forceinline__ float scatter32(float xi, float vx, float vy, float vz, float u, float w,
                                           float &nx, float &ny, float &nz)
{
    const float den = fmaf(-2.0f * xi, u, 1.0f + xi);
    const float mu = __fdividef(fmaf(-2.0f, u, 1.0f + xi), den);
    const float om = __fdividef(2.0f * u * (1.0f - xi), den);
    const float sc = sqrtf(fmaxf(om * (2.0f - om), 0.0f));
    const float v2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
    float d0 = 0.0f, d1 = 0.0f, d2 = 1.0f;
    if (v2 > 0.0f) {
        const float r = rsqrtf(v2);
        d0 = vx * r; d1 = vy * r; d2 = vz * r;
    }
    const float sg = d2 >= 0.0f ? 1.0f : -1.0f;
    const float a = -1.0f / (sg + d2);
    const float b = d0 * d1 * a;
    float sn, cs;
    __sincosf(kTwoPiF * w, &sn, &cs);
    float x = fmaf(mu, d0, sc * fmaf(cs, fmaf(sg * d0 * d0, a, 1.0f), sn * b));
    float y = fmaf(mu, d1, sc * fmaf(cs, sg * b, sn * fmaf(d1 * d1, a, sg)));
    float z = fmaf(mu, d2, sc * fmaf(cs, -sg * d0, -sn * d1));
    const float g = fmaf(x, x, fmaf(y, y, z * z));
    float r = rsqrtf(g);
    r = r * fmaf(-0.5f * g, r * r, 1.5f);
    nx = x * r; ny = y * r; nz = z * r;
    return mu;
}

// Energy of the new electron of an ionisation from the remainder
// rest = eps - I: uniform share u * rest (w = 0), or the inverse of the
// distribution with density proportional to 1 / (1 + (x/w)^2) on
// [0, rest/2] (Opal, Peterson and Beaty, J. Chem. Phys. 55, 4100, 1971).
__device__ __forceinline__ double ionisation_share64(double w, double rest, double u)
{
    return w <= 0.0 ? u * rest : w * tan(u * atan(rest / (2.0 * w)));
}

__device__ __forceinline__ float ionisation_share32(float w, float rest, float u)
{
    return w <= 0.0f ? u * rest : w * tanf(u * atanf(rest / (2.0f * w)));
}

// The new electron of an ionisation (mixed precision): its share of the
// remainder rest = eps - I and its velocity in an isotropic direction, from
// the collision's second random block.  Returned as (vx, vy, vz, share); out
// of line, so that the step's inlined code carries one Philox block, not two.
static __device__ __noinline__ float4 new_electron32(uint64_t seed, int aval, uint64_t uid,
                                                     uint32_t flight, float rest, float split_w)
{
    const uint4 w2 = draw(seed, aval, uid, flight, 1u);
    const float es = ionisation_share32(split_w, rest, u01f(w2.x));
    float sx, sy, sz;
    isotropic32(u01f(w2.y), u01f(w2.z), sx, sy, sz);
    const float ss = sqrtf(kTwoAccelF * es);
    return make_float4(ss * sx, ss * sy, ss * sz, es);
}

// Store the birth record of a new electron in queue slot s: position and
// time are the parent's at the ionising collision (read from the parent),
// energy, velocity and id from the child record.
template <class E, class C>
__device__ __forceinline__ void store_birth(const RunParams &p, int64_t s, const E &parent,
                                            const C &c)
{
    parent.position(p, p.x0[s], p.y0[s], p.z0[s], p.t0[s]);
    p.e0[s] = (double)c.e;
    p.bvx[s] = (double)c.vx; p.bvy[s] = (double)c.vy; p.bvz[s] = (double)c.vz;
    p.belem[s] = parent.birth_elem();  // a new electron starts in its parent's element
    p.uid[s] = c.uid;
    p.aval[s] = parent.aval;
    p.status[s] = 0;
}

// Below-threshold test of an inelastic level in FP64 from the FP32 velocity.
// Kept out of line so that the compiler cannot hoist this rare test (it is
// reached only inside the FP32 margin) into every flight: FP64 instructions
// issue at 1/64 of the FP32 rate on GB300.
static __device__ __noinline__ bool below_threshold64(float vx, float vy, float vz, double thr)
{
    const double e64 = ((double)vx * vx + (double)vy * vy + (double)vz * vz) * kInvTwoAccel;
    return e64 < thr;
}

// The FP64 time-limit decision of a flight that ends near t_max: x = the
// flight time, truncated to reach t_max exactly if T + ot + dt > t_max
// (T = *t_base); y = 1 if truncated.  Out of line for the same reason: nvcc
// turns a short rarely-taken branch into predicated code that issues on
// every flight.
static __device__ __noinline__ float2 time_cut64(const double *t_base, float ot, float dt,
                                                 double t_max)
{
    const double T = *t_base;
    if (T + (double)(ot + dt) > t_max)
        return make_float2(fmaxf((float)((t_max - T) - (double)ot), 0.0f), 1.0f);
    return make_float2(dt, 0.0f);
}

// FP64 boundary test of the position base + o (same role as above: only
// reached when the FP32 pre-test falls inside its margin).
template <int FK>
static __device__ __noinline__ int boundary_confirm64(const double *xb, const double *yb,
                                                      const double *zb, float ox, float oy,
                                                      float oz, double gap, double wire_r2,
                                                      double tube_r2, double lo0, double lo1,
                                                      double lo2, double hi0, double hi1,
                                                      double hi2)
{
    const double x = *xb + (double)ox, y = *yb + (double)oy, z = *zb + (double)oz;
    if (FK == GT_FIELD_PLATE) {
        if (z >= gap) return GT_ST_ANODE;
        if (z < 0.0) return GT_ST_CATHODE;
    } else if (FK == GT_FIELD_COAX) {
        const double r2 = x * x + y * y;
        if (r2 <= wire_r2) return GT_ST_WIRE;
        if (r2 >= tube_r2) return GT_ST_TUBE;
    } else if (FK == GT_FIELD_GRID) {
        const double r2 = x * x + y * y;
        if (wire_r2 > 0.0 && r2 <= wire_r2) return GT_ST_WIRE;
        if (x < lo0 || x > hi0 || y < lo1 || y > hi1 || z < lo2 || z > hi2)
            return GT_ST_OUT_OF_MAP;
    }
    return 0;
}

// FP32 boundary status of a mixed-precision position (the crossing search):
// plate limits zg (anode) and zc (cathode) as offsets from the FP64 base,
// other kinds from the FP32 position (px + ox, ...).
template <int FK>
__device__ __forceinline__ int outside32(const DevField &f, float zg, float zc, float x, float y,
                                         float z)
{
    if (FK == GT_FIELD_PLATE) {
        if (z >= zg) return GT_ST_ANODE;
        if (z < zc) return GT_ST_CATHODE;
    } else if (FK == GT_FIELD_COAX) {
        const float r2 = x * x + y * y;
        if (r2 <= (float)f.wire_r2) return GT_ST_WIRE;
        if (r2 >= (float)f.tube_r2) return GT_ST_TUBE;
    } else if (FK == GT_FIELD_GRID) {
        const float r2 = x * x + y * y;
        if (f.wire_r2 > 0.0 && r2 <= (float)f.wire_r2) return GT_ST_WIRE;
        if (x < (float)f.origin[0] || x > (float)f.hi[0] || y < (float)f.origin[1] ||
            y > (float)f.hi[1] || z < (float)f.origin[2] || z > (float)f.hi[2])
            return GT_ST_OUT_OF_MAP;
    } else if (FK == GT_FIELD_MESH) {
        const float r2 = x * x + y * y;
        if (f.wire_r2 > 0.0 && r2 <= (float)f.wire_r2) return GT_ST_WIRE;
        if (mesh_find32(f, x, y, z, -1, 0.0f) < 0) return GT_ST_OUT_OF_MAP;
    }
    return 0;
}

// --------------------------------------------------- induced signal
// Shockley-Ramo: an electron moving from r_a to r_b induces
// phi_w(r_b) - phi_w(r_a) (units of e) on the readout electrode, phi_w its
// weighting potential; the signal of a time bin is that difference between
// the electron's positions at the bin's edges (or its birth and end).
__device__ __forceinline__ double weighting64(const RunParams &p, double x, double y, double z)
{
    const DevField &f = p.field;
    if (p.signal_kind == GT_W_PLATE) return z * f.inv_gap;
    if (p.signal_kind == GT_W_COAX) return (0.5 * log(x * x + y * y) - f.ln_tube) * f.inv_ln_ab;
    if (f.kind == GT_FIELD_MESH) {  // GT_W_MAP on a mesh: linear in the element
        const int t = mesh_find64(f, x, y, z, -1, 0.0);
        return t < 0 ? 0.0 : mesh_value64(f.tet64 + kMeshRec * (int64_t)t, 3, x, y, z);
    }
    // GT_W_MAP: trilinear interpolation of the nodes' 4th component
    const double q[3] = {x, y, z};
    const int n[3] = {f.nx, f.ny, f.nz};
    int i[3];
    double w[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double g = (q[d] - f.origin[d]) * f.inv_spacing[d];
        int k = (int)floor(g);
        k = k < 0 ? 0 : (k > n[d] - 2 ? n[d] - 2 : k);
        i[d] = k;
        w[d] = g - k;
    }
    double phi = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int di = c & 1, dj = (c >> 1) & 1, dk = (c >> 2) & 1;
        const double wt = (di ? w[0] : 1.0 - w[0]) * (dj ? w[1] : 1.0 - w[1]) *
                          (dk ? w[2] : 1.0 - w[2]);
        const float4 e = __ldg(f.grid + (((int64_t)(i[2] + dk) * f.ny + (i[1] + dj)) * f.nx +
                                         (i[0] + di)));
        phi += wt * (double)e.w;
    }
    return phi;
}

// Index of the first bin edge t0 + j dt after time t (0 before the window).
__device__ __forceinline__ int signal_next(const RunParams &p, double t)
{
    const double x = (t - p.signal_t0) / p.signal_dt;
    if (!(x >= 0.0)) return 0;
    return x >= (double)p.signal_bins ? p.signal_bins + 1 : (int)floor(x) + 1;
}

// Adds phi_b - phi_last to bin `next - 1` (if any) of avalanche `aval`.
__device__ __forceinline__ void signal_add(const RunParams &p, int aval, int next, double d)
{
    if (next >= 1 && next <= p.signal_bins)
        atomicAdd(p.signal + (int64_t)aval * p.signal_bins + (next - 1), d);
}

// ============================================================ FP64 electron
struct Fp64Electron {
    static constexpr bool kTwoPhase = false;
    // New electron produced by an ionising collision (the parent supplies
    // its position and time).
    struct ChildT {
        double e, vx, vy, vz;
        uint64_t uid;
    };

    double x, y, z, t, vx, vy, vz;
    double plate_e;

    __device__ __forceinline__ void bind(const Tables &) {}
    uint32_t nf, nreal, nnull;
    int status;
    int aval;
    uint64_t uid;
    int64_t slot;
    int sg_next;       // induced signal: next bin edge
    double sg_phi;     // weighting potential at the last edge (or birth)

    __device__ __forceinline__ void signal_start(const RunParams &p)
    {
        if (!p.signal_bins) return;
        sg_next = signal_next(p, t);
        sg_phi = sg_next >= 1 ? weighting64(p, x, y, z) : 0.0;
    }

    // Bin edges passed by the step from (x0.., v0..) at ts to te.
    __device__ void signal_step(const RunParams &p, double x0, double y0, double z0, double vx0,
                                double vy0, double vz0, double ax, double ay, double az,
                                double ts, double te)
    {
        while (sg_next <= p.signal_bins) {
            const double tb = p.signal_t0 + (double)sg_next * p.signal_dt;
            if (tb > te) return;
            const double sx = x, sy = y, sz = z, svx = vx, svy = vy, svz = vz;
            x = x0; y = y0; z = z0; vx = vx0; vy = vy0; vz = vz0;
            move(p, ax, ay, az, tb - ts);
            const double ph = weighting64(p, x, y, z);
            x = sx; y = sy; z = sz; vx = svx; vy = svy; vz = svz;
            signal_add(p, aval, sg_next, ph - sg_phi);
            sg_phi = ph;
            ++sg_next;
        }
    }

    // The electron ends (or is parked): the part of its current bin.
    __device__ __forceinline__ void signal_end(const RunParams &p) const
    {
        if (p.signal_bins) signal_add(p, aval, sg_next, weighting64(p, x, y, z) - sg_phi);
    }

    __device__ __forceinline__ void position(const RunParams &, double &ox_, double &oy_,
                                             double &oz_, double &ot_) const
    {
        ox_ = x; oy_ = y; oz_ = z; ot_ = t;
    }

    template <int FK, bool GEO = true>
    __device__ void load_birth(const RunParams &p, int64_t s)
    {
        slot = s;
        x = p.x0[s]; y = p.y0[s]; z = p.z0[s]; t = p.t0[s];
        vx = p.bvx[s]; vy = p.bvy[s]; vz = p.bvz[s];
        uid = p.uid[s];
        aval = p.aval[s];
        plate_e = p.aval_field ? p.aval_field[aval] : p.field.e0;
        nf = nreal = nnull = 0;
        status = 0;
        if (GEO) signal_start(p);
    }

    template <int FK>
    __device__ __forceinline__ int check_start(const RunParams &p)
    {
        status = boundary64<FK>(p.field, x, y, z);
        return status ? EV_RETIRE : EV_NONE;
    }

    // Exact motion over dt with the acceleration a (and the field's B).
    __device__ __forceinline__ void move(const RunParams &p, double ax, double ay, double az,
                                         double dt)
    {
        if (!p.field.has_b) {
            x = x + vx * dt + 0.5 * ax * dt * dt;
            y = y + vy * dt + 0.5 * ay * dt * dt;
            z = z + vz * dt + 0.5 * az * dt * dt;
            vx += ax * dt; vy += ay * dt; vz += az * dt;
        } else {
            double dx, dy, dz;
            lorentz_step<double>(p.field.w, ax, ay, az, dt, vx, vy, vz, dx, dy, dz);
            x += dx; y += dy; z += dz;
        }
    }

    // A flight of length dt in p.substeps equal sub-steps, the field
    // evaluated at the start of each; with p.crossing a sub-step that leaves
    // the volume ends at its first boundary crossing (bisection on the exact
    // motion to 2^-60 of the sub-step; for the plate without B the vertex of
    // z(t) catches a sub-step that leaves and returns).  Moves the electron,
    // returns its boundary status (0 inside) and updates t_end when the
    // electron leaves before the flight's end.
    template <int FK>
    __device__ int fly_steps(const RunParams &p, double dt, double ex, double ey, double ez,
                             double &t_end)
    {
        const int ns = p.substeps > 1 ? p.substeps : 1;
        const double h = ns > 1 ? dt / ns : dt;
        for (int sub = 0; sub < ns; ++sub) {
            if (sub > 0) field64<FK>(p.field, plate_e, x, y, z, ex, ey, ez);
            const double ax = -kAccel * ex, ay = -kAccel * ey, az = -kAccel * ez;
            const double x0 = x, y0 = y, z0 = z, vx0 = vx, vy0 = vy, vz0 = vz;
            move(p, ax, ay, az, h);
            int st = boundary64<FK>(p.field, x, y, z);
            double tc = h;
            if (FK == GT_FIELD_PLATE && p.crossing && !p.field.has_b && az != 0.0) {
                const double tv = -vz0 / az;
                if (tv > 0.0 && tv < h) {
                    const int sv = boundary64<FK>(p.field, x0 + vx0 * tv + 0.5 * ax * tv * tv,
                                                  y0 + vy0 * tv + 0.5 * ay * tv * tv,
                                                  z0 + vz0 * tv + 0.5 * az * tv * tv);
                    if (sv) {
                        st = sv;
                        tc = tv;
                    }
                }
            }
            const double te = sub == ns - 1 ? t_end : t + (sub + 1) * h;  // this step's end
            if (p.crossing && st) {
                double lo = 0.0, hi = tc;
                for (int it = 0; it < 60; ++it) {
                    const double mid = 0.5 * (lo + hi);
                    x = x0; y = y0; z = z0; vx = vx0; vy = vy0; vz = vz0;
                    move(p, ax, ay, az, mid);
                    if (boundary64<FK>(p.field, x, y, z))
                        hi = mid;
                    else
                        lo = mid;
                }
                x = x0; y = y0; z = z0; vx = vx0; vy = vy0; vz = vz0;
                move(p, ax, ay, az, hi);
                t_end = t + sub * h + hi;
                if (p.signal_bins)
                    signal_step(p, x0, y0, z0, vx0, vy0, vz0, ax, ay, az, t + sub * h, t_end);
                return boundary64<FK>(p.field, x, y, z);
            }
            if (p.signal_bins)
                signal_step(p, x0, y0, z0, vx0, vy0, vz0, ax, ay, az, t + sub * h, te);
            if (st) {
                if (sub < ns - 1) t_end = te;
                return st;
            }
        }
        return 0;
    }

    // One flight and its collision (Fig. 2: "Find E field and add random
    // time step", "Collision?", "ionisation or attachment?").  (PHYS is
    // ignored: the FP64 step always handles every gas.)
    template <int FK, bool PHYS = true, bool GEO = true>
    __device__ __forceinline__ int fly(const RunParams &p, const Tables &tb, ChildT &ch)
    {
        if (nf == 0xFFFFFFFFu) {
            status = GT_ST_FLIGHT_LIMIT;
            return EV_RETIRE;
        }
        const uint32_t flight = nf;
        const uint4 w = draw(p.seed, aval + p.aval_base, uid, flight, 0u);
        double ex, ey, ez;
        field64<FK>(p.field, plate_e, x, y, z, ex, ey, ez);
        const double ax = -kAccel * ex, ay = -kAccel * ey, az = -kAccel * ez;
        double nu = p.gas.nu_max, dt;
        bool pseudo = false;
        if (p.majorant == GT_MAJORANT_BANDED) {
            // the rate bound over the energies reachable within the window
            const double eps0 = (vx * vx + vy * vy + vz * vz) * kInvTwoAccel;
            const double tau = p.window / __ldg(p.gas.band64 + band_index64(p.gas, eps0));
            double lo, hi;
            reach64(p.field.has_b, p.field_emax, eps0, vx, vy, vz, ex, ey, ez, tau, lo, hi);
            nu = p.gas.bands_monotone
                     ? __ldg(p.gas.band64 + band_index64(p.gas, hi))
                     : band_range_max(p.gas.band64, p.gas.n_bands, band_index64(p.gas, lo),
                                      band_index64(p.gas, hi));
            dt = -log(u01d(w.x)) / nu;
            if (dt >= tau) {
                dt = tau;
                pseudo = true;
            }
        } else {
            dt = -log(u01d(w.x)) * p.gas.inv_nu_max;
        }
        bool timed = false;
        if (p.t_max > 0.0 && t + dt > p.t_max) {
            dt = p.t_max - t;
            timed = true;
        }
        double t_end = timed ? p.t_max : t + dt;
        int st;
        if (p.substeps > 1 || p.crossing || p.signal_bins) {
            st = fly_steps<FK>(p, dt, ex, ey, ez, t_end);
        } else {
            move(p, ax, ay, az, dt);
            st = boundary64<FK>(p.field, x, y, z);
        }
        t = t_end;
        nf = flight + 1u;
        if (st) {
            status = st;
            return EV_RETIRE;
        }
        if (timed) {
            status = GT_ST_TIME;
            return EV_RETIRE;
        }
        if (pseudo) return EV_NONE;  // the window ended before a collision
        const double eps = (vx * vx + vy * vy + vz * vz) * kInvTwoAccel;
        int lvl = select_level<double, double>(tb.cum64, p.gas.n_levels, p.gas.n_nodes,
                                                p.gas.inv_d_eps, eps, u01d(w.y) * nu);
        if (lvl >= 0 && tb.type[lvl] != GT_LEVEL_ELASTIC && eps < tb.thr[lvl]) lvl = -1;
        if (lvl < 0) {
            ++nnull;
            return EV_NONE;
        }
        tb.tally[lvl * blockDim.x + threadIdx.x] += 1u;
        const int type = tb.type[lvl];
        if (type == GT_LEVEL_ATTACHMENT) {  // captured: the electron ends here
            status = GT_ST_ATTACHED;
            return EV_RETIRE;
        }
        double nx, ny, nz;
        const double xi = p.gas.any_aniso ? level_xi64(p.gas, lvl, eps) : 0.0;
        if (xi == 0.0)
            isotropic64(u01d(w.z), u01d(w.w), nx, ny, nz);
        else
            scatter64(xi, vx, vy, vz, u01d(w.z), u01d(w.w), nx, ny, nz);
        double eps_new;
        int ev = EV_NONE;
        if (type == GT_LEVEL_ELASTIC) {
            const double sp = sqrt(vx * vx + vy * vy + vz * vz);
            const double cchi = sp > 0.0 ? (vx * nx + vy * ny + vz * nz) / sp : 0.0;
            eps_new = eps * (1.0 - p.gas.recoil * (1.0 - cchi));
        } else {
            eps_new = eps - tb.thr[lvl];
            if (type == GT_LEVEL_IONISATION) {
                const uint4 w2 = draw(p.seed, aval + p.aval_base, uid, flight, 1u);
                const double es = ionisation_share64(p.gas.split_w, eps_new, u01d(w2.x));
                eps_new = eps_new - es;
                double sx, sy, sz;
                isotropic64(u01d(w2.y), u01d(w2.z), sx, sy, sz);
                const double ss = sqrt(kTwoAccel * es);
                ch.e = es;
                ch.vx = ss * sx; ch.vy = ss * sy; ch.vz = ss * sz;
                ch.uid = child_uid(uid, flight);
                ev = EV_CHILD;
            }
        }
        const double sp = sqrt(kTwoAccel * eps_new);
        vx = sp * nx; vy = sp * ny; vz = sp * nz;
        ++nreal;
        if (p.coll_limit && nreal >= p.coll_limit) {
            status = GT_ST_COLL_LIMIT;
            return ev | EV_RETIRE;
        }
        return ev;
    }

    template <int FK>
    __device__ __forceinline__ void round_end(const RunParams &) {}
    __device__ __forceinline__ uint32_t level0_count() const { return 0u; }
    __device__ __forceinline__ int birth_elem() const { return -1; }

    __device__ void write_end(const RunParams &p) const
    {
        p.x1[slot] = x; p.y1[slot] = y; p.z1[slot] = z; p.t1[slot] = t;
        p.e1[slot] = (vx * vx + vy * vy + vz * vz) * kInvTwoAccel;
        p.status[slot] = status;
        p.nflight[slot] = nf;
    }

    template <int FK, bool GEO = true>
    __device__ void save(const RunParams &p, const Stack &s, int64_t i)
    {
        if (GEO) signal_end(p);  // the part so far; restore() starts again from here
        s.x[i] = x; s.y[i] = y; s.z[i] = z; s.t[i] = t;
        s.vx[i] = vx; s.vy[i] = vy; s.vz[i] = vz;
        s.nf[i] = nf; s.nreal[i] = nreal; s.uid[i] = uid; s.slot[i] = slot;
    }

    template <int FK, bool GEO = true>
    __device__ void restore(const RunParams &p, const Stack &s, int64_t i, int av)
    {
        x = s.x[i]; y = s.y[i]; z = s.z[i]; t = s.t[i];
        vx = s.vx[i]; vy = s.vy[i]; vz = s.vz[i];
        nf = s.nf[i]; nreal = s.nreal[i]; uid = s.uid[i]; slot = s.slot[i];
        aval = av;
        plate_e = p.aval_field ? p.aval_field[aval] : p.field.e0;
        nnull = 0;
        status = 0;
        if (GEO) signal_start(p);
    }
};

// ===================================================== mixed-precision electron
// The step is split in two so that a warp can handle its lanes' real
// collisions together: advance() makes one free flight and the null test
// against the interpolated total rate; a lane that meets a real collision
// keeps its random words and table position (a Pending record, local to
// one collision round) until collide() selects the level and scatters.
// Each electron still takes exactly the sequence flight, collision,
// flight, ... with the same random numbers.
// Speed after an elastic collision that turns the direction from v to the
// unit vector n (cos chi = mu when `given`, else from v and n), with the
// recoil factor r: |v'| = |v| sqrt(1 - x), x = r (1 - cos chi), scaled on
// the speed itself; a round trip through the energy would multiply by
// (2a)_f32 * (1/2a)_f32 != 1 at every collision and drift.
// |v| = v2 / sqrt(v2) from the hardware rsqrt with one Newton step in
// residual form, r + r h with h = 1/2 - v2 r^2 / 2 from an FMA: within ~2 ulp
// and unbiased (a refinement factor rounded near 1.0 biases the speed by
// ~1e-8 per collision).  Then |v'| = |v| - |v| d with
// d = x/2 + x^2/8 = 1 - sqrt(1 - x) to O(x^3) (x <= 2 recoil ~ 5e-5), one
// FMA: multiplying by a factor rounded just below 1.0 would bias it by
// ~3e-10 per collision (a float32 emulation of both forms; this one is
// unbiased).
__device__ __forceinline__ float elastic_speed32(float vx, float vy, float vz, float nx, float ny,
                                                 float nz, bool given, float mu, float recoil)
{
    const float v2 = vx * vx + vy * vy + vz * vz;
    float r = rsqrtf(v2);
    r = fmaf(r, fmaf(-0.5f * v2 * r, r, 0.5f), r);
    const float cchi = given ? mu : (vx * nx + vy * ny + vz * nz) * r;
    const float x = recoil * (1.0f - cchi);
    const float vm = v2 * r, d = fmaf(0.125f * x, x, 0.5f * x);
    return v2 > 0.f ? fmaf(-vm, d, vm) : 0.f;
}

struct MixedElectron {
    static constexpr bool kTwoPhase = true;
    struct ChildT {
        float e, vx, vy, vz;
        uint64_t uid;
    };
    struct Pending {
        float R;          // u1 * majorant
        float f;          // fraction within table interval k
        int k;
        uint32_t w2, w3;  // direction words
        bool real;
    };

    // The FP64 absolute position and time at the last flush live in the
    // thread's shared-memory slot (b[0], b[S], b[2S], b[3S], S = blockDim),
    // not in registers: they are read only at flushes, ionisations and the
    // rare FP64 confirmations.
    double *b;
    float ox, oy, oz, ot;    // FP32 offsets since the last flush
    float vx, vy, vz;        // FP32 velocity
    float px, py, pz;        // FP32 copy of (X, Y, Z) for field and pre-tests
    float zhi, zlo, tlim;    // pre-test limits for the offsets (see flush)
    float plate_e;
    uint32_t nf, nreal, nnull;
    uint32_t n0;             // real collisions of the straight-line elastic path (level 0)
    int status;
    int aval;
    bool timed;
    uint64_t uid;
    int64_t slot;
    int sg_next;             // induced signal: next bin edge
    double sg_phi;           // weighting potential at the last edge (or birth)
    float sg_toff;           // time offset of the next edge (slightly early)
    int elem;                // MESH: the element holding the position (-1: unknown)

    __device__ __forceinline__ void bind(const Tables &tb) { b = tb.base + threadIdx.x; }

    // Field at the current position.  On a mesh, the element found by the
    // last boundary test holds the position (searched once for a new electron).
    template <int FK>
    __device__ __forceinline__ void efield(const RunParams &p, float &ex, float &ey, float &ez)
    {
        if (FK == GT_FIELD_MESH) {
            const float x = px + ox, y = py + oy, z = pz + oz;
            if (elem < 0) elem = mesh_find32(p.field, x, y, z, -1, -1.0f);
            if (elem < 0) {  // the FP32 position's bin missed: search in FP64
                const unsigned S = blockDim.x;
                elem = mesh_find64(p.field, b[0] + (double)ox, b[S] + (double)oy,
                                   b[2 * S] + (double)oz, -1, 0.0);
            }
            if (elem < 0) {
                ex = ey = ez = 0.f;
                return;
            }
            mesh_field32(p.field.tet32 + (kMeshRec / 4) * (int64_t)elem, x, y, z, ex, ey, ez);
        } else {
            field32<FK>(p.field, plate_e, px + ox, py + oy, pz + oz, ex, ey, ez);
        }
    }

    // FP32 offset time at which the next bin edge may come (an FP32
    // pre-test; the edge itself is placed in FP64).
    __device__ __forceinline__ void signal_limit(const RunParams &p)
    {
        if (!p.signal_bins || sg_next > p.signal_bins) {
            sg_toff = 3.0e38f;
            return;
        }
        const float g = (float)(p.signal_t0 + (double)sg_next * p.signal_dt - b[3 * blockDim.x]);
        sg_toff = g - (fabsf(g) * 1e-6f + 1e-12f);
    }

    __device__ __forceinline__ void signal_start(const RunParams &p)
    {
        if (!p.signal_bins) return;
        double x, y, z, t;
        position(p, x, y, z, t);
        sg_next = signal_next(p, t);
        sg_phi = sg_next >= 1 ? weighting64(p, x, y, z) : 0.0;
        signal_limit(p);
    }

    // Bin edges passed by the step that started at offsets (so.., sot) with
    // velocity sv and acceleration a and ended now (at t_max if `at_tmax`).
    __device__ void signal_step(const RunParams &p, float sox, float soy, float soz, float sot,
                                float svx, float svy, float svz, float ax, float ay, float az,
                                bool at_tmax)
    {
        const unsigned S = blockDim.x;
        const double ts = b[3 * S] + (double)sot;
        const double te = at_tmax ? p.t_max : b[3 * S] + (double)ot;
        while (sg_next <= p.signal_bins) {
            const double tb = p.signal_t0 + (double)sg_next * p.signal_dt;
            if (tb > te) break;
            const float h = (float)(tb - ts);
            float dx, dy, dz;
            if (!p.field.has_b) {
                dx = h * fmaf(0.5f * h, ax, svx);
                dy = h * fmaf(0.5f * h, ay, svy);
                dz = h * fmaf(0.5f * h, az, svz);
            } else {
                float wx = svx, wy = svy, wz = svz;
                lorentz_step<float>(p.field.w_f, ax, ay, az, h, wx, wy, wz, dx, dy, dz);
            }
            const double ph = weighting64(p, b[0] + (double)(sox + dx), b[S] + (double)(soy + dy),
                                          b[2 * S] + (double)(soz + dz));
            signal_add(p, aval, sg_next, ph - sg_phi);
            sg_phi = ph;
            ++sg_next;
        }
        signal_limit(p);
    }

    // The electron ends (or is parked): the part of its current bin.
    __device__ __forceinline__ void signal_end(const RunParams &p) const
    {
        if (!p.signal_bins) return;
        double x, y, z, t;
        position(p, x, y, z, t);
        signal_add(p, aval, sg_next, weighting64(p, x, y, z) - sg_phi);
    }

    __device__ __forceinline__ void position(const RunParams &, double &x_, double &y_,
                                             double &z_, double &t_) const
    {
        const unsigned S = blockDim.x;
        x_ = b[0] + (double)ox; y_ = b[S] + (double)oy;
        z_ = b[2 * S] + (double)oz; t_ = b[3 * S] + (double)ot;
    }

    // Fold the FP32 offsets into the FP64 state and refresh the FP32
    // pre-test limits: an offset beyond a limit is re-tested in FP64.
    template <int FK>
    __device__ __forceinline__ void flush(const RunParams &p)
    {
        const unsigned S = blockDim.x;
        set_base<FK>(p, b[0] + (double)ox, b[S] + (double)oy, b[2 * S] + (double)oz,
                     b[3 * S] + (double)ot);
        if (p.signal_bins) signal_limit(p);
    }

    // New FP64 base (X, Y, Z, T) with zero offsets, and the pre-test limits.
    template <int FK>
    __device__ __forceinline__ void set_base(const RunParams &p, double X, double Y, double Z,
                                             double T)
    {
        const unsigned S = blockDim.x;
        b[0] = X; b[S] = Y; b[2 * S] = Z; b[3 * S] = T;
        ox = oy = oz = ot = 0.f;
        if (FK == GT_FIELD_COAX || FK == GT_FIELD_GRID || FK == GT_FIELD_MESH) {
            px = (float)X; py = (float)Y;
        }
        if (FK == GT_FIELD_GRID || FK == GT_FIELD_MESH) pz = (float)Z;
        if (FK == GT_FIELD_PLATE) {
            const float hi = (float)(p.field.gap - Z), lo = -(float)Z;
            zhi = hi - (fabsf(hi) * 1e-6f + 1e-12f);
            zlo = lo + (fabsf(lo) * 1e-6f + 1e-12f);
        }
        if (p.t_max > 0.0) {
            const float g = (float)(p.t_max - T);
            tlim = g - (fabsf(g) * 1e-6f + 1e-12f);
        } else {
            tlim = 3.0e38f;
        }
    }

    template <int FK, bool GEO = true>
    __device__ void load_birth(const RunParams &p, int64_t s)
    {
        slot = s;
        vx = (float)p.bvx[s]; vy = (float)p.bvy[s]; vz = (float)p.bvz[s];
        uid = p.uid[s];
        aval = p.aval[s];
        plate_e = (float)(p.aval_field ? p.aval_field[aval] : p.field.e0);
        nf = nreal = nnull = n0 = 0;
        status = 0;
        timed = false;
        elem = FK == GT_FIELD_MESH ? p.belem[s] : -1;
        set_base<FK>(p, p.x0[s], p.y0[s], p.z0[s], p.t0[s]);
        if (GEO) signal_start(p);
    }

    template <int FK>
    __device__ __forceinline__ int check_start(const RunParams &p)
    {
        status = boundary64<FK>(p.field, p.x0[slot], p.y0[slot], p.z0[slot]);
        return status ? EV_RETIRE : EV_NONE;
    }

    // FP32 pre-test with a margin, then the FP64 boundary test of X + ox.
    template <int FK>
    __device__ __forceinline__ int boundary(const RunParams &p)
    {
        bool maybe;
        if (FK == GT_FIELD_UNIFORM) {
            return 0;
        } else if (FK == GT_FIELD_MESH) {
            // inside for sure when an element holds the FP32 position with a
            // margin (the cached element first); else decided in FP64
            const DevField &f = p.field;
            const float rx = px + ox, ry = py + oy, rz = pz + oz;
            const bool near = (rx * rx + ry * ry <= f.wire_r2_hi_f) || (rx < f.box_lo_f[0]) ||
                              (rx > f.box_hi_f[0]) || (ry < f.box_lo_f[1]) ||
                              (ry > f.box_hi_f[1]) || (rz < f.box_lo_f[2]) || (rz > f.box_hi_f[2]);
            if (!near) {
                int t = elem >= 0 ? mesh_walk32(f, rx, ry, rz, elem, 1.0f) : -1;
                if (t < 0) t = mesh_find32(f, rx, ry, rz, -1, 1.0f);
                if (t >= 0) {
                    elem = t;
                    return 0;
                }
            }
            const unsigned S = blockDim.x;
            const double x = b[0] + (double)ox, y = b[S] + (double)oy, z = b[2 * S] + (double)oz;
            if (f.wire_r2 > 0.0 && x * x + y * y <= f.wire_r2) return GT_ST_WIRE;
            const int t = mesh_find_mixed(f, x, y, z, rx, ry, rz, elem);
            if (t < 0) return GT_ST_OUT_OF_MAP;
            elem = t;
            return 0;
        } else if (FK == GT_FIELD_PLATE) {
            maybe = (oz >= zhi) || (oz < zlo);
        } else {
            const DevField &f = p.field;
            const float rx = px + ox, ry = py + oy;
            const float r2 = rx * rx + ry * ry;
            maybe = (r2 <= f.wire_r2_hi_f);
            if (FK == GT_FIELD_COAX) {
                maybe |= (r2 >= f.tube_r2_lo_f);
            } else {
                const float rz = pz + oz;
                maybe |= (rx < f.box_lo_f[0]) || (rx > f.box_hi_f[0]) || (ry < f.box_lo_f[1]) ||
                         (ry > f.box_hi_f[1]) || (rz < f.box_lo_f[2]) || (rz > f.box_hi_f[2]);
            }
        }
        if (!maybe) return 0;
        const DevField &f = p.field;
        const unsigned S = blockDim.x;
        return boundary_confirm64<FK>(b, b + S, b + 2 * S, ox, oy, oz, f.gap, f.wire_r2,
                                      f.tube_r2, f.origin[0], f.origin[1], f.origin[2], f.hi[0],
                                      f.hi[1], f.hi[2]);
    }

    // Exact motion of the FP32 offsets over dt with the acceleration a
    // (no_b: the run has no magnetic field; z_only: the field is along z, so
    // ax = ay = 0 and x, y move uniformly; both known at compile time).
    __device__ __forceinline__ void move(const RunParams &p, float ax, float ay, float az, float dt,
                                         bool no_b = false, bool z_only = false)
    {
        float dx, dy, dz;
        if (no_b || !p.field.has_b) {
            const float h = 0.5f * dt;
            if (z_only) {
                dx = dt * vx;
                dy = dt * vy;
            } else {
                dx = dt * fmaf(h, ax, vx);
                dy = dt * fmaf(h, ay, vy);
                vx = fmaf(ax, dt, vx); vy = fmaf(ay, dt, vy);
            }
            dz = dt * fmaf(h, az, vz);
            vz = fmaf(az, dt, vz);
        } else {
            lorentz_step<float>(p.field.w_f, ax, ay, az, dt, vx, vy, vz, dx, dy, dz);
        }
        ox += dx; oy += dy; oz += dz;
    }

    // A flight of length dt in p.substeps equal sub-steps (the field at the
    // start of each), with the first boundary crossing located in FP64
    // (crossing64) when p.crossing is set.  Returns the boundary status; on
    // a crossing the FP64 base moves to the crossing point and time.
    template <int FK, int MODE = 0>
    __device__ int fly_steps(const RunParams &p, float dt, float ex, float ey, float ez)
    {
        // MODE 2: exact crossings, MODE 3: induced signals, each alone in a
        // run without B or sub-steps, known at compile time; MODE 0: any run
        constexpr bool XONLY = MODE == 2, SONLY = MODE == 3, ONE = XONLY || SONLY;
        const bool sig = SONLY || (!XONLY && p.signal_bins != 0);
        const bool cross = XONLY || (!SONLY && p.crossing != 0);
        const int ns = ONE ? 1 : (p.substeps > 1 ? p.substeps : 1);
        const bool zonly = ONE && (FK == GT_FIELD_PLATE || FK == GT_FIELD_UNIFORM);
        const float h = ns > 1 ? dt / (float)ns : dt;
        const unsigned S = blockDim.x;
        for (int sub = 0; sub < ns; ++sub) {
            if (sub > 0) efield<FK>(p, ex, ey, ez);
            const float ax = -kAccelF * ex, ay = -kAccelF * ey, az = -kAccelF * ez;
            const float sox = ox, soy = oy, soz = oz, sot = ot, svx = vx, svy = vy, svz = vz;
            move(p, ax, ay, az, h, ONE, zonly);
            ot += h;
            int st = boundary<FK>(p);
            float tc = h;
            if (FK == GT_FIELD_PLATE && cross && (ONE || !p.field.has_b) && az != 0.0f) {
                // a sub-step that leaves the gap and returns: the vertex of z(t)
                const float tv = -svz / az;
                if (tv > 0.0f && tv < h) {
                    const float zv = soz + tv * fmaf(0.5f * tv, az, svz);
                    if (zv >= zhi || zv < zlo) {
                        const int sv = boundary_confirm64<FK>(b, b + S, b + 2 * S, sox, soy, zv,
                                                              p.field.gap, 0.0, 0.0, 0.0, 0.0,
                                                              0.0, 0.0, 0.0, 0.0);
                        if (sv) {
                            st = sv;
                            tc = tv;
                        }
                    }
                }
            }
            if (cross && st) {
                // first crossing within (0, tc], by bisection on the FP32
                // motion of the offsets (2^-32 of tc: below FP32 resolution);
                // the point found is on the surface to FP32 rounding
                const float zg = FK == GT_FIELD_PLATE ? (float)(p.field.gap - b[2 * S]) : 0.0f;
                const float zc = FK == GT_FIELD_PLATE ? (float)(-b[2 * S]) : 0.0f;
                float lo = 0.0f, hi = tc;
                for (int it = 0; it < 32; ++it) {
                    const float mid = 0.5f * (lo + hi);
                    ox = sox; oy = soy; oz = soz; vx = svx; vy = svy; vz = svz;
                    move(p, ax, ay, az, mid, ONE, zonly);
                    if (outside32<FK>(p.field, zg, zc, px + ox, py + oy,
                                      FK == GT_FIELD_PLATE ? oz : pz + oz))
                        hi = mid;
                    else
                        lo = mid;
                }
                ox = sox; oy = soy; oz = soz; vx = svx; vy = svy; vz = svz;
                move(p, ax, ay, az, hi, ONE, zonly);
                ot = sot + hi;
                timed = false;  // the electron left before the time limit
                if (sig && ot >= sg_toff)
                    signal_step(p, sox, soy, soz, sot, svx, svy, svz, ax, ay, az, false);
                const int sc = outside32<FK>(p.field, zg, zc, px + ox, py + oy,
                                             FK == GT_FIELD_PLATE ? oz : pz + oz);
                return sc ? sc : st;
            }
            if (sig && ot >= sg_toff)
                signal_step(p, sox, soy, soz, sot, svx, svy, svz, ax, ay, az,
                            timed && sub == ns - 1);
            if (st) return st;
        }
        return 0;
    }

    // One free flight and the real/null decision (Fig. 2 "Find E field and
    // add random time step", "Collision?").  Returns EV_RETIRE or EV_NONE;
    // fills `pd` (pd.real) for a real collision.  GEO = true also builds
    // the sub-steps and exact crossings of fly_steps().
    // MAJ = 1 builds the step for runs with the banded majorant, band bounds
    // that rise with energy, an elastic level 0, no magnetic field and the
    // field held over the flight (the common case), without the run-time
    // tests of the others; MAJ = 2 the same with exact crossings and neither
    // sub-steps nor signals; MAJ = 3 with induced signals and neither
    // sub-steps nor crossings.
    template <int FK, bool GEO, int MAJ = 0>
    __device__ __forceinline__ int advance(const RunParams &p, const Tables &tb, Pending &pd)
    {
        pd.real = false;
        if (nf == 0xFFFFFFFFu) {
            status = GT_ST_FLIGHT_LIMIT;
            return EV_RETIRE;
        }
        const uint4 w = draw_rk(p.rk, aval + p.aval_base, uid, nf, 0u);
        float ex, ey, ez;
        efield<FK>(p, ex, ey, ez);
        const float ax = -kAccelF * ex, ay = -kAccelF * ey, az = -kAccelF * ez;
        float nu = p.gas.nu_max_f, dt;
        bool pseudo = false;
        if (MAJ >= 1 || p.majorant == GT_MAJORANT_BANDED) {
            // the rate bound over the energies reachable within the window
            const bool mono = MAJ >= 1 || p.gas.bands_monotone;
            const float eps0 = (vx * vx + vy * vy + vz * vz) * kInvTwoAccelF;
            const float tau = __fdividef(p.window_f, tb.band32[band_index32(p.gas, eps0)]);
            float lo, hi;
            reach32<FK>(MAJ >= 1 ? 0 : p.field.has_b, MAJ >= 1 ? 0.0f : p.field_emax_f, eps0, vx,
                        vy, vz, ex, ey, ez, plate_e, tau, lo, hi, !mono);
            nu = mono
                     ? tb.band32[band_index32(p.gas, hi)]
                     : band_range_max(tb.band32, p.gas.n_bands, band_index32(p.gas, lo),
                                      band_index32(p.gas, hi));
            dt = -__fdividef(__logf(u01f(w.x)), nu);
            if (dt >= tau) {
                dt = tau;
                pseudo = true;
            }
        } else {
            dt = -__logf(u01f(w.x)) * p.gas.inv_nu_max_f;
        }
        if (ot + dt >= tlim) {  // near the time limit: decide in FP64
            const float2 c = time_cut64(b + 3 * blockDim.x, ot, dt, p.t_max);
            dt = c.x;
            timed = c.y != 0.0f;
        }
        int st;
        if (GEO && (MAJ >= 2 || p.substeps > 1 || p.crossing || p.signal_bins)) {
            st = fly_steps<FK, MAJ>(p, dt, ex, ey, ez);
        } else {
            move(p, ax, ay, az, dt, MAJ >= 1, FK == GT_FIELD_PLATE || FK == GT_FIELD_UNIFORM);
            ot += dt;
            st = boundary<FK>(p);
        }
        ++nf;
        if (st | (int)timed) {
            status = st ? st : GT_ST_TIME;
            return EV_RETIRE;
        }
        // null test against the interpolated total rate, as straight-line
        // code; a pseudo-flight (the window ended before a collision) takes
        // no test
        const float eps = (vx * vx + vy * vy + vz * vz) * kInvTwoAccelF;
        const float R = u01f(w.y) * nu;
        const float xk = eps * p.gas.inv_d_eps_f;
        const float tk = __fadd_rd(fminf(xk, p.gas.lastk_f), 8388608.0f);
        const int k = __float_as_int(tk) - 0x4B000000;
        const float f = fminf(xk, p.gas.last_x_f) - (tk - 8388608.0f);
        const int L = p.gas.n_levels;
        const float *c0 = tb.cum32 + k * tb.stride32 + (L - 1);
        const float top = fmaf(f, c0[tb.stride32] - c0[0], c0[0]);
        const bool real = !pseudo && R < top;
        pd.real = real;
        pd.R = R;
        pd.k = k;
        pd.f = f;
        pd.w2 = w.z;
        pd.w3 = w.w;
        nnull += (!pseudo && !real) ? 1u : 0u;
        return EV_NONE;
    }

    // The pending real collision (Fig. 2 "Collision is ionisation or
    // attachment?"): level selection, threshold guard, isotropic scattering.
    // PHYS = false builds the collision of a gas with isotropic levels, no
    // attachment and a uniform ionisation split (the basic gas) without the
    // code of the general case; PHYS = true handles every gas.
    template <int FK, bool PHYS, int MAJ = 0>
    __device__ __forceinline__ int collide(const RunParams &p, const Tables &tb, Pending &pd,
                                           ChildT &ch)
    {
        pd.real = false;
        const float *c0 = tb.cum32 + pd.k * tb.stride32;
        // most real collisions are elastic (level 0 when it is the elastic
        // level): when every colliding lane's R lies below the level-0 sum,
        // the warp skips the search
        const bool lvl0 = (MAJ >= 1 || p.gas.level0_elastic) &&
                          __all_sync(__activemask(), pd.R < fmaf(pd.f, c0[tb.stride32] - c0[0], c0[0]));
        if (lvl0 && !(PHYS && p.gas.any_aniso)) {
            // the common case as straight-line code: every colliding lane of
            // the warp scatters elastically and isotropically on level 0
            ++n0;
            float nx, ny, nz;
            isotropic32(u01f(pd.w2), u01f(pd.w3), nx, ny, nz);
            const float sp = elastic_speed32(vx, vy, vz, nx, ny, nz, false, 0.0f,
                                             p.gas.recoil_f);
            vx = sp * nx; vy = sp * ny; vz = sp * nz;
            ++nreal;
            if (p.coll_limit && nreal >= p.coll_limit) {
                status = GT_ST_COLL_LIMIT;
                return EV_RETIRE;
            }
            return EV_NONE;
        }
        // the energy at the collision (the velocity has not changed since the flight)
        const float eps = (vx * vx + vy * vy + vz * vz) * kInvTwoAccelF;
        const int lvl = lvl0 ? 0 : select_below_total32(c0, tb.stride32, p.gas.n_levels, pd.f, pd.R);
        const int type = tb.type[lvl];
        if (type != GT_LEVEL_ELASTIC) {
            const float th = tb.thr_f[lvl];
            if (eps < th * (1.0f + 1e-6f)) {
                if (eps < th * (1.0f - 1e-6f) || below_threshold64(vx, vy, vz, tb.thr[lvl])) {
                    ++nnull;
                    return EV_NONE;
                }
            }
        }
        tb.tally[lvl * blockDim.x + threadIdx.x] += 1u;
        if (PHYS && type == GT_LEVEL_ATTACHMENT) {  // captured: the electron ends here
            status = GT_ST_ATTACHED;
            return EV_RETIRE;
        }
        float nx, ny, nz;
        float sp;
        int ev = EV_NONE;
        float xi = 0.0f, mu = 0.0f;
        if (PHYS && p.gas.any_aniso) {
            const float sc = tb.screen_f[lvl];
            xi = sc > 0.0f ? __fdividef(eps, eps + sc) : tb.xi0_f[lvl];
        }
        if (xi != 0.0f)
            mu = scatter32(xi, vx, vy, vz, u01f(pd.w2), u01f(pd.w3), nx, ny, nz);
        else
            isotropic32(u01f(pd.w2), u01f(pd.w3), nx, ny, nz);
        if (type == GT_LEVEL_ELASTIC) {
            sp = elastic_speed32(vx, vy, vz, nx, ny, nz, xi != 0.0f, mu, p.gas.recoil_f);
        } else {
            float eps_new = fmaxf(eps - tb.thr_f[lvl], 0.0f);
            if (type == GT_LEVEL_IONISATION) {
                const uint32_t flight = nf - 1u;
                const float4 c = new_electron32(p.seed, aval + p.aval_base, uid, flight, eps_new,
                                                PHYS ? p.gas.split_w_f : 0.0f);
                eps_new = eps_new - c.w;
                ch.e = c.w;
                ch.vx = c.x; ch.vy = c.y; ch.vz = c.z;
                ch.uid = child_uid(uid, flight);
                ev = EV_CHILD;
            }
            sp = sqrt_nr(kTwoAccelF * eps_new);
        }
        vx = sp * nx; vy = sp * ny; vz = sp * nz;
        ++nreal;
        if (p.coll_limit && nreal >= p.coll_limit) {
            status = GT_ST_COLL_LIMIT;
            return ev | EV_RETIRE;
        }
        return ev;
    }

    // Flight and collision in one call (plain mode).
    template <int FK, bool PHYS = true, bool GEO = true>
    __device__ __forceinline__ int fly(const RunParams &p, const Tables &tb, ChildT &ch)
    {
        Pending pd;
        const int ev = advance<FK, GEO>(p, tb, pd);
        if (ev || !pd.real) return ev;
        return collide<FK, PHYS>(p, tb, pd, ch);
    }

    template <int FK>
    __device__ __forceinline__ void round_end(const RunParams &p)
    {
        flush<FK>(p);
    }
    __device__ __forceinline__ int birth_elem() const { return elem; }
    __device__ __forceinline__ uint32_t level0_count() const { return n0; }

    __device__ void write_end(const RunParams &p) const
    {
        double x, y, z, t;
        position(p, x, y, z, t);
        p.x1[slot] = x; p.y1[slot] = y; p.z1[slot] = z;
        p.t1[slot] = timed ? p.t_max : t;
        p.e1[slot] = ((double)vx * vx + (double)vy * vy + (double)vz * vz) * kInvTwoAccel;
        p.status[slot] = status;
        p.nflight[slot] = nf;
    }

    template <int FK, bool GEO = true>
    __device__ void save(const RunParams &p, const Stack &s, int64_t i)
    {
        if (GEO) signal_end(p);  // the part so far; restore() starts again from here
        position(p, s.x[i], s.y[i], s.z[i], s.t[i]);
        s.vx[i] = vx; s.vy[i] = vy; s.vz[i] = vz;
        s.nf[i] = nf; s.nreal[i] = nreal; s.uid[i] = uid; s.slot[i] = slot;
    }

    template <int FK, bool GEO = true>
    __device__ void restore(const RunParams &p, const Stack &s, int64_t i, int av)
    {
        vx = (float)s.vx[i]; vy = (float)s.vy[i]; vz = (float)s.vz[i];
        nf = s.nf[i]; nreal = s.nreal[i]; uid = s.uid[i]; slot = s.slot[i];
        aval = av;
        plate_e = (float)(p.aval_field ? p.aval_field[aval] : p.field.e0);
        nnull = n0 = 0;
        status = 0;
        timed = false;
        elem = -1;
        set_base<FK>(p, s.x[i], s.y[i], s.z[i], s.t[i]);
        if (GEO) signal_start(p);
    }
};

}  // namespace gt

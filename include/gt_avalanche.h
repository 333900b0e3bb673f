/*
 * gt_avalanche.h -- C ABI of the GB300 microscopic avalanche transport library.
 *
 * The library transports electrons collision by collision through a gas in
 * an electric (and optionally uniform magnetic) field and multiplies them by
 * ionisation: the AvalancheMicroscopic method of "Accelerating Garfield++
 * with CUDA" (arXiv:2509.15377, Sec. 2, Fig. 2).  Each electron takes
 * null-collision free flights dt = -ln(u)/nu_max (Skullerud's technique,
 * cited in Sec. 1) in the field at the start of the flight; its kinetic
 * energy indexes tabulated per-level collision rates (Magboltz-style tables,
 * Sec. 1 and Sec. 4); a real or null collision is chosen; an elastic,
 * excitation or ionising collision is applied with isotropic scattering; an
 * ionisation appends a new electron to a device work queue ("stack
 * processing", Sec. 2).  An electron stops when it leaves the volume, reaches
 * its time limit or its collision limit ("Position is valid?", Fig. 2; status
 * codes, Sec. 2).  The run returns, per electron, its start and end point
 * (the endpoint record of Sec. 3.2) and, per avalanche, the number of
 * electrons and the collision tallies.
 *
 * Units everywhere: cm, ns, eV, V/cm, T; rates in 1/ns.
 *
 * Conventions of every entry point:
 *   - returns GT_OK (0) or a negative GT_ERR_* code; no exception or abort
 *     crosses the ABI; gt_strerror() names the code;
 *   - "host" pointers are read during the call only; "device" pointers are
 *     CUDA device memory of the context's device owned by the caller, which
 *     must stay valid until the call returns;
 *   - the library owns only the context and what it uploads into it (the
 *     rate table and the field constants); every output buffer, the work
 *     space and the stream belong to the caller;
 *   - avalanche_run is stream-ordered on the caller's stream and returns
 *     after that stream has finished the run (it reads back a small status
 *     block); it is not safe to call concurrently on one context.
 */
#ifndef GT_AVALANCHE_H
#define GT_AVALANCHE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GT_ABI_VERSION 4
#define GT_MAX_LEVELS 32 /* collision levels per gas table */

/* ---- return codes ---------------------------------------------------- */
#define GT_OK 0
#define GT_ERR_ARG (-1)            /* invalid argument (null pointer, size, range) */
#define GT_ERR_STATE (-2)          /* gas table or field not set up */
#define GT_ERR_WORKSPACE (-3)      /* work space too small or misaligned */
#define GT_ERR_QUEUE_OVERFLOW (-4) /* more electrons than endpoint capacity: the
                                      stored ones are complete, the rest dropped */
#define GT_ERR_TIMEOUT (-5)        /* a bounded wait or the run's time budget ran
                                      out: the result is partial */
#define GT_ERR_CUDA (-6)           /* a CUDA runtime call failed */
#define GT_ERR_NO_DEVICE (-7)      /* no usable CUDA device */
#define GT_ERR_UNSUPPORTED (-8)    /* combination not implemented */
#define GT_ERR_HOST_MEMORY (-9)    /* a host allocation failed (e.g. a very large mesh) */

/* ---- electron status codes (endpoint.status; non-zero = finished) ---- */
#define GT_ST_ACTIVE 0        /* not finished (only in a partial result) */
#define GT_ST_ANODE 1         /* PLATE: z >= gap */
#define GT_ST_CATHODE 2       /* PLATE: z < 0 */
#define GT_ST_WIRE 3          /* COAX/GRID/MESH: x^2 + y^2 <= wire_r^2 */
#define GT_ST_TUBE 4          /* COAX: x^2 + y^2 >= tube_r^2 */
#define GT_ST_OUT_OF_MAP 5    /* GRID: outside the map box; MESH: in no element */
#define GT_ST_TIME 6          /* reached t_max */
#define GT_ST_COLL_LIMIT 7    /* reached coll_limit real collisions */
#define GT_ST_FLIGHT_LIMIT 8  /* 2^32 - 1 flights */
#define GT_ST_ATTACHED 9      /* captured by an attachment collision (Fig. 2
                                 "ionisation or attachment?") */

/* ---- enumerations ---------------------------------------------------- */
#define GT_LEVEL_ELASTIC 0    /* energy x (1 - recoil (1 - cos chi)) */
#define GT_LEVEL_EXCITATION 1 /* energy - threshold */
#define GT_LEVEL_IONISATION 2 /* energy - threshold shared with a new electron
                                 in an isotropic direction (see split_w) */
#define GT_LEVEL_ATTACHMENT 3 /* the electron is captured: it ends at the
                                 collision with status GT_ST_ATTACHED */

#define GT_FIELD_UNIFORM 0 /* E = (0, 0, -e0) everywhere, no boundary */
#define GT_FIELD_PLATE 1   /* E = (0, 0, -E_k) between z = 0 and z = gap */
#define GT_FIELD_COAX 2    /* E = V / (r ln(b/a)) r-hat, wire radius a, tube b */
#define GT_FIELD_GRID 3    /* trilinear interpolation of a regular float4 map */
#define GT_FIELD_MESH 4    /* linear interpolation on a tetrahedral mesh (FEM-like map) */

#define GT_FP64 0  /* every step in FP64 */
#define GT_MIXED 1 /* FP32 kinematics, table and scattering; FP64 position and
                      time accumulation and FP64 threshold/boundary decisions */

#define GT_BATCHED 0 /* all avalanches in one persistent kernel with a global
                        electron queue */
#define GT_PLAIN 1   /* one avalanche at a time, one transport launch per
                        generation followed by stack compaction (the
                        structure of the paper's GPU port, Sec. 2) */

typedef struct gt_ctx gt_ctx;

/* ---- gas table (Sec. 1 and Sec. 4: tabulated cross-sections) ----------
 * rate[k * n_levels + j] is the collision rate of level j at the node energy
 * k * d_eps (1/ns, >= 0); between nodes the rates are interpolated linearly,
 * beyond the last node the last node is used.  nu_max <= 0 selects
 * (1 + 1e-6) * max_k sum_j rate; a given nu_max must be >= that maximum.
 * The upload also tabulates, per energy band, the largest total rate (the
 * band's largest node value: rates are linear between nodes), for runs with
 * the banded majorant. */
typedef struct {
    int32_t n_levels;          /* 1..GT_MAX_LEVELS */
    int32_t n_nodes;           /* >= 2 */
    double d_eps;              /* eV, > 0 */
    const int32_t *level_type; /* host [n_levels] GT_LEVEL_* */
    const double *threshold;   /* host [n_levels] eV lost (excitation, ionisation) */
    const double *rate;        /* host [n_nodes * n_levels] 1/ns */
    double recoil;             /* 2 m / M for elastic recoil loss, in [0, 0.5) */
    double nu_max;             /* 1/ns */
    double band_width;         /* eV per energy band of the banded majorant,
                                  rounded to whole nodes; 0 = 1 eV */
    /* Angular model per level (NULL = isotropic for all levels): the
     * anisotropy is xi = xi0[j] where screen[j] == 0, else
     * xi = eps / (eps + screen[j]); xi = 0 scatters isotropically in the lab
     * frame, otherwise the deflection chi from the incident direction has
     * the screened-Coulomb density (1 - xi^2) / (2 (1 - xi cos chi)^2) in
     * cos chi and a uniform azimuth. */
    const double *xi0;         /* host [n_levels] in (-1, 1), or NULL */
    const double *screen;      /* host [n_levels] eV >= 0, or NULL */
    double split_w;            /* ionisation sharing: 0 = the new electron takes a
                                  uniform share of eps - I; > 0 = a share on
                                  [0, (eps - I)/2] with density proportional to
                                  1 / (1 + (x / split_w)^2) (eV) */
} gt_gas;

/* ---- field and geometry (Fig. 2 "Find E field"; Sec. 3.1 field maps) -- */
typedef struct {
    int32_t kind;              /* GT_FIELD_* */
    double e0;                 /* UNIFORM |E|; PLATE default |E| (V/cm) */
    double gap;                /* PLATE anode position (cm) */
    double wire_r, tube_r;     /* COAX radii; GRID wire radius (0 = none) (cm) */
    double voltage;            /* COAX wire voltage (V) */
    double b[3];               /* uniform magnetic field (T) */
    int32_t nx, ny, nz;        /* GRID nodes, each >= 2 */
    double origin[3];          /* GRID position of node (0,0,0) (cm) */
    double spacing[3];         /* GRID node spacing (cm) */
    const float *grid;         /* GRID device [nz][ny][nx] float4 (Ex, Ey, Ez, -),
                                  16-byte aligned; kept by pointer, must stay
                                  valid while runs use this field */
    /* MESH (Sec. 3.1: field maps are finite-element solutions on tetrahedral
     * meshes, searched for the element of a point).  Host arrays, copied by
     * field_setup (the caller keeps ownership and may free them after the
     * call).  A point's element is a closed tetrahedron that holds it (every
     * barycentric coordinate >= 0); the field and the weighting potential are
     * interpolated linearly from the element's four nodes.  A point in no
     * element is out of the map (GT_ST_OUT_OF_MAP); wire_r > 0 adds the wire
     * test of GRID.  Every element must have a non-zero volume.  field_setup
     * builds the element records and a uniform bin structure over the mesh's
     * box for the element search. */
    int64_t n_mesh_nodes;      /* MESH nodes, >= 4 */
    int64_t n_tets;            /* MESH elements, 1 .. 2^26 */
    const double *mesh_nodes;  /* MESH host [n_mesh_nodes][3] positions (cm) */
    const int32_t *mesh_tets;  /* MESH host [n_tets][4] node indices */
    const float *mesh_values;  /* MESH host [n_mesh_nodes][4] (Ex, Ey, Ez, weighting
                                  potential) at the nodes (V/cm; 1) */
} gt_field;

/* ---- one run --------------------------------------------------------- */
typedef struct {
    int64_t n_primaries;
    int32_t n_avalanches;
    int32_t primaries_on_device;  /* 0: the arrays below are host memory and are
                                     copied inside the run; 1: device memory */
    const double *x, *y, *z, *t, *e;  /* [n_primaries] position, time, energy */
    const double *dx, *dy, *dz;       /* [n_primaries] unit direction */
    const int32_t *aval;              /* [n_primaries] avalanche in [0, n_avalanches) */
    const uint64_t *uid;              /* [n_primaries] electron ids, unique */
    const double *aval_field;         /* PLATE: [n_avalanches] |E| per avalanche
                                         (same memory kind), or NULL for e0 */
    uint64_t seed;
    double t_max;                     /* ns, <= 0: none */
    uint32_t coll_limit;              /* real collisions per electron, 0: none */
    int32_t precision;                /* GT_FP64 / GT_MIXED */
    int32_t mode;                     /* GT_BATCHED / GT_PLAIN */
    int32_t block;                    /* threads per CTA, 0 = default */
    int32_t refill_period;            /* BATCHED: steps between refills of idle lanes
                                         from the queue (and FP32-to-FP64 flushes):
                                         FP64 one flight per step, MIXED one
                                         collision round per step; 0 = default */
    int32_t grid;                     /* BATCHED: CTAs, 0 = one per SM */
    uint64_t size_limit;              /* BATCHED: max electrons per avalanche,
                                         further secondaries dropped; 0 = none */
    double spin_limit_ms;             /* longest wait without queue progress, 0 =
                                         60 s; exceeded -> GT_ERR_TIMEOUT */
    double time_limit_ms;             /* whole-run budget, 0 = 600 s */
    int32_t debug_flags;              /* GT_DEBUG_*, 0 in normal use */
    int32_t flights_per_phase;        /* BATCHED MIXED: a collision round lets each
                                         lane fly up to this many flights until it
                                         meets a real collision, then the warp
                                         applies its lanes' collisions together;
                                         0 = default (1 with the banded majorant,
                                         6 with the global one) */
    int32_t majorant;                 /* GT_MAJORANT_GLOBAL / GT_MAJORANT_BANDED */
    int32_t aval_base;                /* >= 0: number of this run's avalanche 0 in a
                                         larger workload.  Avalanches are independent
                                         (Sec. 2), and the random streams are chosen
                                         by the workload's avalanche number
                                         aval[i] + aval_base (it enters the Philox
                                         counter), so a run of avalanches
                                         [a0, a1) of a workload with aval_base = a0
                                         (and the workload's electron ids) transports
                                         exactly those avalanches of the whole run:
                                         a workload can be split over GPUs and the
                                         parts gathered.  Every per-avalanche array
                                         (aval_field, electrons, tallies, signal,
                                         endpoint aval) stays indexed by aval[i]. */
    double majorant_window;           /* banded: window factor c, 0 = 2 */
    int32_t substeps;                 /* field evaluations per flight: <= 1 holds
                                         the field of the flight's start (Sec. 2
                                         reading); n > 1 splits every flight into
                                         n equal sub-steps, each in the field at
                                         its own start (at most 4096) */
    int32_t crossing;                 /* 0: an electron that leaves the volume ends
                                         at the point after its (sub-)step; 1: at
                                         its first boundary crossing, found by
                                         bisection on the exact motion of the
                                         (sub-)step (to 2^-60 of it); for the plate
                                         without B a step that leaves and returns
                                         is caught at the vertex of z(t) */
    /* Induced signal (Shockley-Ramo theorem): with signal_kind != GT_W_NONE
     * and signal_bins > 0, out->signal[a][j] receives the charge (in units
     * of e) that the electrons of avalanche a induce on the readout electrode
     * during [signal_t0 + j signal_dt, signal_t0 + (j+1) signal_dt): for each
     * electron the change of the electrode's weighting potential phi_w
     * between its positions at the bin's edges (or its birth and end inside
     * the bin).  Positive when electrons move towards the electrode. */
    int32_t signal_kind;              /* GT_W_* */
    int32_t signal_bins;
    double signal_t0;                 /* ns */
    double signal_dt;                 /* ns, > 0 */
} gt_run;

/* Readout electrodes for induced signals (their weighting potentials). */
#define GT_W_NONE 0
#define GT_W_PLATE 1 /* PLATE anode: phi_w = z / gap */
#define GT_W_COAX 2  /* COAX (or GRID, MESH) wire: phi_w = ln(r / tube_r) / ln(wire_r / tube_r) */
#define GT_W_MAP 3   /* GRID: trilinear interpolation of the map's 4th component; MESH: the
                        nodes' 4th value, linear in the element */

/* Majorant of the null-collision flights.
 * GLOBAL: dt = -ln(u)/nu_max with one nu_max for all energies (Skullerud).
 * BANDED: per flight, with tau = c / (largest rate of the band holding the
 * current energy), the energy can change by at most
 * D = |E| (|v| tau + a tau^2 / 2) during tau (the field's work bound; B
 * does no work), so the largest rate over the bands covering
 * [eps - D, eps + D] bounds the true rate along the whole flight; dt is drawn
 * with that bound, and a flight longer than tau stops at tau without a
 * collision test (a memoryless restart).  Both are exact; BANDED needs
 * several times fewer flights per real collision when the rates vary with
 * energy.  Flight counts include the stopped flights; null tallies count
 * only rejected collision tests. */
#define GT_MAJORANT_GLOBAL 0
#define GT_MAJORANT_BANDED 1

/* Fault injection for tests: reserve one queue slot that is never filled,
 * so every waiting worker eventually gives up after spin_limit_ms and the
 * run returns GT_ERR_TIMEOUT (the GPU context stays usable). */
#define GT_DEBUG_UNFILLED_SLOT 1

/* ---- outputs (caller-owned device arrays) ------------------------------
 * Endpoint slot i holds one electron: slots [0, n_primaries) are the
 * primaries in input order, later slots the electrons created by ionisation
 * in completion order (the order of those is not reproducible; sort by uid).
 * This is the record of GetElectronEndpoint (Sec. 3.2): start x0..e0, end
 * x1..e1 and the status, plus the avalanche, the id and the flight count. */
typedef struct {
    int64_t capacity;                 /* slots in every per-electron array */
    double *x0, *y0, *z0, *t0, *e0;   /* [capacity] start */
    double *x1, *y1, *z1, *t1, *e1;   /* [capacity] end */
    int32_t *status;                  /* [capacity] GT_ST_* */
    int32_t *aval;                    /* [capacity] */
    uint64_t *uid;                    /* [capacity] */
    uint32_t *n_flight;               /* [capacity] flights (real + null) */
    uint64_t *electrons;              /* [n_avalanches] electrons stored */
    uint64_t *tallies;                /* [n_avalanches][n_levels + 1] real
                                         collisions per level, then null ones */
    double *signal;                   /* [n_avalanches][signal_bins] induced charge
                                         (set to 0 by the run), or NULL without
                                         a signal */
} gt_endpoints;

/* ---- run summary (host, filled by avalanche_run) ---------------------- */
typedef struct {
    int64_t n_endpoints;      /* slots written */
    int64_t n_dropped;        /* secondaries not stored (capacity or size_limit) */
    uint64_t real_collisions; /* elastic + excitation + ionisation */
    uint64_t null_collisions; /* flights ending in a null collision */
    uint64_t flights;         /* all flights, including the final ones */
    double transport_ms;      /* GPU time of the transport kernel(s), CUDA
                                 events on the run's stream */
    int32_t launches;         /* kernels launched by the run */
    int32_t iterations;       /* PLAIN: generations summed over avalanches */
    int32_t status;           /* same value as the return code */
    int32_t block, refill_period, grid; /* launch shape actually used */
    int32_t flights_per_phase;
    int32_t pad;
} gt_stats;

/* ---- entry points ---------------------------------------------------- */

/* ABI version of the loaded library (GT_ABI_VERSION). */
int gt_abi_version(void);

/* Human-readable name of a return code.  Static string, never NULL. */
const char *gt_strerror(int code);

/* sizeof of gt_gas, gt_field, gt_run, gt_endpoints and gt_stats, written to
 * sizes[0..4] (n >= 5), so that bindings can check their struct layouts.
 * Needs no device. */
int gt_abi_sizes(size_t *sizes, int n);

/* Text of the last CUDA failure seen by this context ("" if none).  Valid
 * until the next call on the context. */
const char *gt_last_cuda_error(gt_ctx *ctx);

/* Create a context on CUDA device `device` (the GPUExclusive run mode and
 * device index of SetRunModeOptions, Sec. 3.2).  *ctx receives the handle.
 * GT_ERR_NO_DEVICE if the device does not exist or is not a GB300-class
 * (sm_103) device this library was built for. */
int gt_create(gt_ctx **ctx, int device);

/* Release the context and everything it uploaded.  NULL is accepted. */
int gt_destroy(gt_ctx *ctx);

/* Upload a gas table (Sec. 3.1: preprocessed once on the host, copied once
 * to the GPU).  Builds the cumulative per-level rate table in FP64 and FP32,
 * nu_max and the per-level constants.  Replaces any previous table.
 * GT_ERR_ARG for a negative rate, a bad size, an unknown level type or a
 * nu_max below the total rate. */
int gas_table_upload(gt_ctx *ctx, const gt_gas *gas);

/* nu_max (1/ns) of the uploaded table. */
int gt_gas_nu_max(gt_ctx *ctx, double *nu_max);

/* Set the field and geometry used by later runs (Sec. 3.1: the field data
 * is transferred once, before the first transport).  The GRID map stays in
 * caller memory and is read by pointer.  A MESH is copied from the host
 * arrays and turned into element records, face neighbours and search bins
 * held by the context (replaced by the next field_setup, freed by
 * gt_destroy).  GT_ERR_ARG for an unknown kind, a non-finite or
 * non-positive size, a node index out of range, an element of zero volume,
 * a face shared by more than two elements or a non-finite nodal value;
 * GT_ERR_CUDA if a device allocation or copy fails. */
int field_setup(gt_ctx *ctx, const gt_field *field);

/* Work-space bytes that avalanche_run needs for `run` with endpoint
 * `capacity`.  The work space is caller-owned device memory, 256-byte
 * aligned; its contents need no initialisation. */
int gt_workspace_bytes(gt_ctx *ctx, const gt_run *run, int64_t capacity, size_t *bytes);

/* Transport every avalanche of `run` to completion (Fig. 2 repeated until
 * no electron is active) and fill `out` and `*stats`.  `stream` is a
 * cudaStream_t (NULL = the legacy default stream).  Returns GT_OK, or
 * GT_ERR_QUEUE_OVERFLOW / GT_ERR_TIMEOUT with a partial but consistent
 * result, or an argument / CUDA error with nothing guaranteed in `out`. */
int avalanche_run(gt_ctx *ctx, const gt_run *run, const gt_endpoints *out, void *workspace,
                  size_t workspace_bytes, void *stream, gt_stats *stats);

/* ---- the batched run without a caller work space ----------------------
 * avalanche_run_static runs exactly like avalanche_run in GT_BATCHED mode,
 * but its scratch memory (queue flags, birth velocities, run header,
 * per-avalanche counters) is a fixed array inside the library, so the call
 * itself allocates nothing: no cudaMalloc, no cudaFree, no host heap.  It
 * is for callers that cannot allocate device memory where they run
 * avalanches: code living inside a framework whose memory manager owns the
 * GPU's memory, or a loop that cannot accept the device synchronisation an
 * allocation or a free may cause.  The paper has no counterpart.
 *
 * Limits: out->capacity <= GT_STATIC_MAX_ELECTRONS and n_avalanches <=
 * GT_STATIC_MAX_AVALANCHES, else GT_ERR_WORKSPACE; primaries must be in
 * device memory (primaries_on_device = 1) and mode GT_BATCHED, else
 * GT_ERR_ARG.  The caller still provides the primaries and every output
 * array, as for avalanche_run.
 *
 * The array (GT_STATIC_SCRATCH_BYTES) is held by every GPU that loads the
 * library, until the process exits.  The first call on a device looks up the
 * array's device address for that device (cudaGetSymbolAddress), which may
 * load the library's device code; make that first call before any stream
 * capture.  All calls on a device share the one array: calls whose runs
 * overlap on the GPU (other streams, other contexts, other threads) race
 * and corrupt each other; serialise them.  Each call clears what must start
 * at zero, so the contents left by the previous call do not matter. */
#define GT_STATIC_MAX_ELECTRONS (1 << 18)
#define GT_STATIC_MAX_AVALANCHES 16384
#define GT_STATIC_SCRATCH_BYTES 8520192 /* ~8.1 MiB */

int avalanche_run_static(gt_ctx *ctx, const gt_run *run, const gt_endpoints *out, void *stream,
                         gt_stats *stats);

/* ---- captured launch graphs ------------------------------------------
 * The device work of one batched run -- zeroing the outputs and the run
 * header, seeding the queue, the persistent transport, the per-avalanche
 * electron counts and the copy of the run's status -- recorded once as a
 * CUDA graph and replayed with one launch.  The run must be GT_BATCHED with
 * primaries in device memory; every replay reads the primaries and writes
 * the outputs at the addresses given to gt_graph_create (the caller may
 * refill the primaries between replays; n_primaries and n_avalanches are
 * fixed).  The graph keeps the run's launch shape.
 *   gt_graph_create   records the graph (nothing runs); errors as
 *                     avalanche_run, GT_ERR_UNSUPPORTED for GT_PLAIN or host
 *                     primaries;
 *   gt_graph_launch   enqueues a replay on `stream` with `seed` (a seed that
 *                     differs from the last one records the graph again and
 *                     updates it in place, tens of microseconds on the host);
 *                     GT_ERR_STATE once gas_table_upload or field_setup has
 *                     run on the context after the graph was created (the
 *                     graph holds the tables of its own setup: create a new
 *                     graph);
 *   gt_graph_stats    waits for the last replay and returns its summary and
 *                     status (as avalanche_run; GT_ERR_STATE before a launch);
 *   gt_graph_destroy  releases it (after its replays have finished).
 * A graph belongs to one context and must not be used from two threads at
 * once; its replays, like runs, must not overlap on the same outputs. */
typedef struct gt_graph gt_graph;

int gt_graph_create(gt_ctx *ctx, const gt_run *run, const gt_endpoints *out, void *workspace,
                    size_t workspace_bytes, gt_graph **graph);
int gt_graph_launch(gt_graph *graph, uint64_t seed, void *stream);
int gt_graph_stats(gt_graph *graph, gt_stats *stats);
int gt_graph_destroy(gt_graph *graph);

/* ---- autotuning of the batched launch shape ---------------------------
 * The batched kernel's throughput depends on the threads per CTA (more
 * resident warps against fewer registers each) and on the flights per
 * round (fewer queue refills and FP64 flushes against lanes idling after
 * their electron finishes).  gt_autotune runs `run` in GT_BATCHED mode (after
 * one warm-up run) and measures real collisions per millisecond of transport
 * kernel time (CUDA events) for the shapes of a coordinate descent: from a
 * middle shape, each dimension in turn takes its best value with the others
 * held, until a whole sweep changes nothing (at most four sweeps; a shape
 * runs at most once; typically 10-14 runs, so a sample large enough to keep
 * the GPU saturated is affordable).  Values: MIXED 512/768/896/1024 threads,
 * refill period 4/8/16/32, flights per phase 1/2/4/6; FP64 128/256/512
 * threads, refill period 8/16/32/64.  A block, refill_period or
 * flights_per_phase set (non-zero) in `run` fixes that dimension.  The
 * fastest shape is remembered by the context for the run's
 * precision, field kind, majorant and kernel build (the basic gas; a gas
 * with anisotropy, attachment or a sharing law; a run with sub-steps,
 * crossings or signals), and used by later runs that leave block /
 * refill_period / flights_per_phase at 0.
 * points (may be NULL) receives up to max_points measurements, *n_points
 * their number; *best the chosen shape.  Errors as avalanche_run; a
 * candidate that fails is skipped. */
typedef struct {
    int32_t block;
    int32_t refill_period;
    int32_t flights_per_phase;
    int32_t pad;
    double real_per_ms;
    double transport_ms;
} gt_tune_point;

int gt_autotune(gt_ctx *ctx, const gt_run *run, const gt_endpoints *out, void *workspace,
                size_t workspace_bytes, void *stream, gt_tune_point *points, int32_t max_points,
                int32_t *n_points, gt_tune_point *best);

/* Observables of a finished run (Sec. 2: gain = electrons at the end of the
 * avalanche / initial electrons), computed on the device from the first
 * n_endpoints slots of `ep` and written as GT_OBS_COUNT doubles to the
 * device array obs:
 *   [0] mean gain: electrons ending with status `collect_status`, averaged
 *       over avalanches with at least one primary, per primary;
 *   [1] standard error of [0];
 *   [2] number of avalanches with at least one primary;
 *   [3] drift velocity sum(z1 - z0) / sum(t1 - t0) (cm/ns) over electrons
 *       ending with `drift_status` (any status if drift_status < 0);
 *   [4] transverse diffusion <(x1-x0)^2 + (y1-y0)^2> / (4 <t1-t0>) (cm^2/ns);
 *   [5] longitudinal diffusion var(z1 - z0) / (2 <t1-t0>) (cm^2/ns);
 *   [6] electrons counted in [3]..[5];
 *   [7] Townsend coefficient ln([0]) / gap (1/cm; 0 unless gap > 0).
 * `n_primaries_per_aval` is a device int32 [n_avalanches] array. */
#define GT_OBS_COUNT 8
int avalanche_observables(gt_ctx *ctx, const gt_endpoints *ep, int64_t n_endpoints,
                          int32_t n_avalanches, const int32_t *n_primaries_per_aval,
                          int32_t collect_status, int32_t drift_status, double gap,
                          double *obs, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GT_AVALANCHE_H */

/*
 * swe.h - C ABI of the GB300 shallow-water step library (libswe.so).
 *
 * One explicit Euler step of a cell-centred finite-volume solver for the 2D
 * shallow-water equations on an unstructured triangle mesh (Zaoui, "A
 * GPU-enabled finite volume solver for large shallow water simulations"):
 *   Sec. 2.1, Eq. 1  state U = (h, hu, hv), physical fluxes G, H, bed slope
 *                    and Manning friction sources;
 *   Sec. 2.2, Eq. 2-4 finite volumes on triangles, the face sum
 *                    sum_k F_k . n_k l_k, explicit Euler update;
 *   Sec. 2.2         HLLC interface fluxes, hydrostatic reconstruction of the
 *                    bed, semi-implicit friction, CFL time step (Courant 0.7);
 *   Sec. 2.3         state and mesh stay on the device; the host only starts
 *                    steps and copies results at the end.
 *   Sec. 3           reflective (wall) boundaries on every boundary edge.
 *
 * Conventions for every call:
 *   - Host pointers are plain host memory (pageable or pinned); the library
 *     copies what it needs and never keeps a caller pointer.
 *   - Cell arrays are indexed in the CALLER's cell order (the order of `tri`).
 *     Any renumbering the library does for locality is internal.
 *   - All work is queued on the CUDA stream given to swe_mesh_create (NULL =
 *     a stream the library creates). Calls that return results to the host
 *     synchronise that stream; swe_run does not.
 *   - Errors are returned as negative swe_status codes, never by abort/trap.
 *     Device-side conditions (NaN, all-dry) latch an error word that the next
 *     synchronising call reports.
 *   - Handles are owned by the caller and freed with the matching destroy.
 *     Destroying a mesh that states still use is allowed: the mesh is freed
 *     when the last of them is destroyed. Handles are not thread-safe.
 */
#ifndef SWE_H
#define SWE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int swe_status;

#define SWE_OK 0
#define SWE_EINVAL (-1)     /* bad argument (null pointer, negative size, bad enum) */
#define SWE_EMESH (-2)      /* bad mesh: node index out of range, zero-area triangle,
                               an edge shared by more than two triangles, empty mesh */
#define SWE_ENOMEM (-3)     /* device or host allocation failed */
#define SWE_ECUDA (-4)      /* a CUDA runtime call failed (no device, launch error) */
#define SWE_ENAN (-5)       /* a non-finite value appeared in the state */
#define SWE_ETIMEOUT (-7)   /* a bounded device-side wait ran out */
#define SWE_EDRY (-8)       /* no wet cell left: the CFL time step is undefined */
#define SWE_ESTATE (-9)     /* call not valid for this handle (e.g. wrong precision) */

/* Arithmetic of the state, the fluxes and the update. */
typedef enum {
  SWE_F64 = 0, /* everything in FP64 (the paper's precision, Sec. 3) */
  SWE_F32 = 1  /* FP32 state and fluxes, compensated per-cell flux sums, FP64 mass
                  integral and FP64 wet/dry depth tests */
} swe_precision;

/* Internal cell numbering (locality of the neighbour gathers). */
typedef enum {
  SWE_ORDER_NONE = 0,    /* keep the caller's order */
  SWE_ORDER_MORTON = 1,  /* Z-order of the cell centroids; edges follow their cells */
  SWE_ORDER_RCM = 2      /* reverse Cuthill-McKee order of the edge-neighbour graph */
} swe_order;

/* Kernel structure of one step. */
typedef enum {
  SWE_KERNEL_AUTO = 0,  /* SWE_KERNEL_TILED; SWE_KERNEL_EDGE for a single mesh in
                           SWE_ORDER_RCM, whose tiles would be thin strips */
  SWE_KERNEL_EDGE = 1,  /* two launches: per-edge fluxes to HBM, then a per-cell gather
                           and update (the paper's two parallel loops, Sec. 2.3) */
  SWE_KERNEL_TILED = 2  /* one launch: each block stages a tile of cells in shared
                           memory, computes every face flux of the tile once, then
                           updates its cells */
} swe_kernel;

typedef struct {
  double g;           /* gravity, m/s^2 (default 9.81) */
  double courant;     /* Courant number (default 0.7, Sec. 2.2) */
  double h_eps;       /* dry threshold in m (default 1e-6): cells at or below it carry
                         no momentum, reconstructed sides at or below it are dry */
  int32_t precision;  /* swe_precision (default SWE_F64) */
  int32_t order;      /* swe_order (default SWE_ORDER_MORTON) */
  int32_t kernel;     /* swe_kernel (default SWE_KERNEL_AUTO) */
  int32_t tile;       /* cells per tile of SWE_KERNEL_TILED; tile / cells_per_thread threads
                         per block must be 32, 64, 128 or 256; 0 = default (512 in
                         FP32 at 2 cells per thread, else 256) */
  int32_t stages;     /* shared-memory pipeline stages of SWE_KERNEL_TILED (2 or 3);
                         0 = default (2) */
  int32_t cells_per_thread;  /* cells each thread updates per tile (1 or 2); 0 = default (2) */
  int32_t halo_schedule;     /* schedule of the SWE_KERNEL_TILED step: 0 = default, a tile's
                                halo cells gathered after the previous tile's face loop;
                                1 = gathered at the start of the previous tile, so the gather
                                overlaps its whole face loop; 2 = pipelined: the cell updates
                                of a tile overlap the face loop of the next one, one block
                                barrier per tile instead of two (two sets of face slots).
                                Which is faster depends on the mesh: a choice for the
                                autotuner. 1 and 2 apply to FP32 meshes with 2 stages whose
                                halo lists fit one entry per thread, and are ignored
                                otherwise. Results are identical. */
  int32_t wait_rounds;       /* bounded device waits of SWE_KERNEL_TILED steps (a block waiting
                                for its tile copies) give up after this many rounds of at most
                                20 us and latch SWE_ETIMEOUT: 0 = default (50,000 rounds,
                                about a second); n > 0 = n rounds; -1 = give up at once, so
                                every step of the mesh ends with SWE_ETIMEOUT (a hook for
                                testing the timeout path: copies already in flight are still
                                waited for before a block exits, and nothing is left
                                running). Other values: SWE_EINVAL. */
  int32_t compensated_depth; /* 1: an SWE_F32 state also keeps, per cell, the FP32 residual of
                                its depth (h + residual is the depth). The Euler update (Eq. 4)
                                of h is then carried exactly up to its final rounding and the
                                rounding error goes to the residual, so updates below half an
                                ulp of h accumulate instead of being lost and the mass is kept
                                over long runs. Faces use h; copy-outs and the mass integral
                                use h + residual. 4 B per cell more in HBM, 8 B more traffic
                                per step. Needs SWE_F32, SWE_KERNEL_TILED (or AUTO), 2 stages
                                and halo_schedule 0; not for swe_grad_record. 0 = off
                                (default); other values: SWE_EINVAL. */
} swe_params;

typedef struct swe_mesh swe_mesh;
typedef struct swe_state swe_state;

/* Fills *p with the defaults listed in swe_params. */
void swe_params_default(swe_params* p);

/* Builds a device-resident mesh from host arrays.
 *   xy       [2*n_nodes] node coordinates (x0, y0, x1, y1, ...), metres.
 *   tri      [3*n_tris]  node ids of each triangle, any orientation (clockwise
 *            triangles are reoriented).
 *   params   numerics and layout; NULL = defaults. Copied.
 *   cuda_stream  a cudaStream_t, or NULL for a library-owned stream.
 * Builds the edges (interior and wall), the geometry of Eq. 3 (areas, unit
 * normals, edge lengths, perimeters) in FP64 on the host, renumbers cells and
 * edges, and uploads everything. Returns SWE_EMESH for an invalid mesh,
 * SWE_EINVAL for bad arguments. *out receives the handle. */
swe_status swe_mesh_create(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tris,
                           const swe_params* params, void* cuda_stream, swe_mesh** out);

/* Host only (no device is touched): the internal cell order swe_mesh_create
 * gives this mesh under `order` (a swe_order), perm[j] = caller index of
 * the cell at internal position j (perm: n_tris entries, caller-owned).
 * SWE_EMESH for an invalid mesh, SWE_EINVAL for bad arguments. */
swe_status swe_cell_order(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tris,
                          int32_t order, int32_t* perm);

/* Builds one device-resident mesh holding n_scenarios independent scenarios
 * (an ensemble): scenario i has the nodes xy[i] (n_nodes[i] of them) and the
 * triangles tri[i] (n_tris[i]), in the formats of swe_mesh_create. The
 * scenarios share no edge and each keeps its own time, CFL time step, step
 * count, error word and mass; one step launch advances all of them (the
 * paper's per-cell parallelism, Sec. 2.3, over the union of their cells).
 * Cell arrays of every other call are the concatenation of the scenarios'
 * cells in scenario order (scenario 0's n_tris[0] cells first). Requires
 * SWE_KERNEL_TILED (or AUTO); SWE_KERNEL_EDGE with n_scenarios > 1 returns
 * SWE_EINVAL. Each scenario is validated as swe_mesh_create validates a
 * mesh; the first invalid one makes the call fail with nothing allocated.
 * swe_mesh_create(...) is this call with n_scenarios = 1. */
swe_status swe_mesh_create_batch(int32_t n_scenarios, const double* const* xy,
                                 const int64_t* n_nodes, const int32_t* const* tri,
                                 const int64_t* n_tris, const swe_params* params,
                                 void* cuda_stream, swe_mesh** out);

/* counts[0..3] = nodes, triangles, edges, wall edges (sums over scenarios). */
swe_status swe_mesh_counts(const swe_mesh* mesh, int64_t* counts);

/* *n_scenarios = scenarios in the mesh; n_tris (may be NULL, else
 * [*n_scenarios] entries, caller-allocated: call once with NULL to size it)
 * receives each scenario's triangle count. */
swe_status swe_mesh_scenarios(const swe_mesh* mesh, int32_t* n_scenarios, int64_t* n_tris);

/* Device bytes held by the mesh. */
swe_status swe_mesh_device_bytes(const swe_mesh* mesh, int64_t* bytes);

void swe_mesh_destroy(swe_mesh* mesh);

/* Creates a state on a mesh from host arrays of n_tris values each, caller order:
 * depth h (m), discharges hu, hv (m^2/s), bed z (m), per-cell Manning n
 * (s/m^{1/3}) or NULL to use manning_const everywhere. Sets t = 0 and computes
 * the first CFL time step (Sec. 2.2, Courant 0.7) from this state. The
 * fields are copied to the device here, once (Sec. 2.3: the state stays on
 * the device between steps). Returns SWE_EDRY if no cell is wet, SWE_ENAN if
 * a value is not finite. */
swe_status swe_state_init(swe_mesh* mesh, const double* h, const double* hu, const double* hv,
                          const double* z, const double* manning, double manning_const,
                          swe_state** out);

/* swe_state_init with DEVICE arrays (FP64, caller order, on the mesh's
 * device; e.g. the data pointers of contiguous float64 torch CUDA tensors):
 * h, hu, hv, z and manning (or NULL and manning_const). cuda_stream is the
 * stream the caller wrote them on (NULL or the mesh's stream: no extra
 * ordering); the library's stream waits for the work queued there so far.
 * Nothing goes through host memory. Synchronises the library's stream before
 * returning, so the caller may reuse the arrays at once. Same results,
 * bitwise, as swe_state_init with the same values. */
swe_status swe_state_init_device(swe_mesh* mesh, const double* h, const double* hu,
                                 const double* hv, const double* z, const double* manning,
                                 double manning_const, void* cuda_stream, swe_state** out);

/* Replaces (h, hu, hv) from host arrays (caller order) and resets t = 0 and
 * the step count; bed and friction stay. The next CFL time step is
 * recomputed from the new state (Sec. 2.2). Arrays in page-locked host
 * memory (cudaHostAlloc, cudaHostRegister) are read by one kernel across
 * the host link; other host memory goes through a device staging buffer.
 * The arrays are no longer used when the call returns. */
swe_status swe_state_set(swe_state* state, const double* h, const double* hu, const double* hv);

/* swe_state_set from FP32 host arrays (caller order), for callers that keep
 * the fields of an SWE_F32 state in FP32: the values are those the state
 * holds (swe_state_set rounds FP64 values to the nearest FP32), so the
 * state equals swe_state_set's with the same values in FP64, in half the
 * bytes. An SWE_F64 state widens them exactly. */
swe_status swe_state_set_f32(swe_state* state, const float* h, const float* hu, const float* hv);

/* swe_state_set with DEVICE arrays (FP64, caller order), ordered after the
 * work queued on cuda_stream as swe_state_init_device is. Synchronises. */
swe_status swe_state_set_device(swe_state* state, const double* h, const double* hu,
                                const double* hv, void* cuda_stream);

/* One explicit Euler step (Eq. 4) with the current CFL time step (no
 * end-time clamp): per face the HLLC flux of the hydrostatically
 * reconstructed states (Sec. 2.2) in the face frame of Eq. 3, per cell the
 * sum over its three faces and the update U - dt / Omega * sum, then the
 * semi-implicit Manning friction (Sec. 2.2) and the CFL time step of the new
 * state (Courant 0.7). Synchronises; *dt_used (may be NULL) receives the
 * step's dt (scenario 0's on an ensemble: every scenario steps with its own
 * CFL dt). */
swe_status swe_step(swe_state* state, double* dt_used);

/* Queues n_steps steps of swe_step (Eq. 4, each with its CFL dt, Sec. 2.2)
 * without an end time and returns without synchronising (device errors are
 * reported by the next synchronising call). Steps are replayed from
 * captured CUDA graphs; the host reads nothing back between them (Sec. 2.3:
 * no transfer during the time loop). n_steps = 0 takes no step and only
 * captures (and uploads) the step graph if the state has none yet, so that
 * the steps of a later call are replayed from its first one. */
swe_status swe_run(swe_state* state, int64_t n_steps);

/* Steps until t == t_end exactly (the simulated end time T_s of the paper's
 * runs, Sec. 3): each step uses min(CFL dt, t_end - t), and the step that
 * reaches t_end sets t = t_end. Synchronises once per chunk of
 * graph-replayed steps. *n_steps (may be NULL) receives the steps taken
 * (scenario 0's). On an ensemble every scenario stops at t_end on its own
 * step count; launches continue until the last one gets there. */
swe_status swe_advance(swe_state* state, double t_end, int64_t* n_steps);

/* Waits for queued work and returns the latched device status. */
swe_status swe_sync(swe_state* state);

/* Copies the state to host arrays in caller order (any pointer may be NULL):
 * the one device-to-host transfer at the end of a run (Sec. 2.3).
 * *t = simulated time (scenario 0's on an ensemble), *mass = sum of area * h
 * in FP64 over every cell. Synchronises. Arrays in page-locked host memory
 * are written by one kernel across the host link; other host memory is
 * written through a device staging buffer. */
swe_status swe_copy_out(const swe_state* state, double* h, double* hu, double* hv, double* t,
                        double* mass);

/* swe_copy_out into FP32 host arrays: exact for an SWE_F32 state (its
 * values are FP32), rounded to the nearest FP32 for an SWE_F64 state. t and
 * mass as in swe_copy_out (FP64). */
swe_status swe_copy_out_f32(const swe_state* state, float* h, float* hu, float* hv, double* t,
                            double* mass);

/* swe_copy_out into DEVICE arrays (FP64, caller order, any may be NULL; t
 * and mass are host scalars as in swe_copy_out). The library's stream first
 * waits for the work queued so far on cuda_stream (the caller's earlier use
 * of the destinations); the call synchronises before returning, so the
 * arrays are ready for any stream. Nothing goes through host memory. */
swe_status swe_copy_out_device(const swe_state* state, double* h, double* hu, double* hv,
                               double* t, double* mass, void* cuda_stream);

/* info[0] = steps taken (scenario 0's), info[1] = cells whose depth went
 * negative and was clipped to 0 (expected 0 under the CFL step), info[2] =
 * latched error bits (both over every scenario). */
swe_status swe_state_info(const swe_state* state, int64_t* info);

/* The CFL time step the next swe_step would use (before any end-time clamp).
 * On an ensemble: scenario 0's (see swe_scenario_info). */
swe_status swe_next_dt(const swe_state* state, double* dt);

/* One scenario of an ensemble (0 <= scenario < n_scenarios, else
 * SWE_EINVAL): its time, mass (sum of area * h over its cells, FP64), steps
 * taken and next CFL time step; any output pointer may be NULL. Returns that
 * scenario's latched status. Synchronises. */
swe_status swe_scenario_info(const swe_state* state, int32_t scenario, double* t, double* mass,
                             int64_t* steps, double* dt_next);

void swe_state_destroy(swe_state* state);

/* ---------------------------------------------------------------------------
 * Gradients through many steps (reverse mode; no counterpart in the paper).
 *
 * The derivative is that of the step of Sec. 2.2 with the time steps held
 * fixed at the values the recorded run used (dt is data, not a function of
 * the state), differentiated piecewise: each wet/dry test, HLLC case and
 * min/max takes the branch the forward step took. A depth clipped at zero
 * (never under the CFL step) is differentiated as if unclipped.
 *
 * Usage: swe_grad_record runs the steps and keeps a tape; swe_grad then
 * computes, for a loss L given by its derivatives with respect to the final
 * state and to the gauge depths, the gradient of L with respect to the
 * initial state, the bed z and Manning's n. swe_grad can be called any
 * number of times on one tape (different seeds). Requires a single-scenario
 * mesh built with SWE_KERNEL_TILED, without ghost cells and without
 * compensated_depth (SWE_ESTATE otherwise). Results are in
 * the mesh precision; FP64 is the reference for accuracy. The adjoint runs
 * on the mesh's tiles: 256-cell tiles (swe_params.tile = 256) give the faster
 * adjoint, since at 512 cells its shared memory fits half as many blocks per
 * SM.
 * ------------------------------------------------------------------------- */
typedef struct swe_tape swe_tape;

/* Advances `state` by n_steps CFL steps (as swe_run does, with no end time)
 * and records: every step's dt, the depth at each of the n_gauges cells
 * gauge_cells[j] (caller indices, repeats allowed) after every step into
 * gauge_h[k * n_gauges + j] for step k = 0 .. n_steps-1 (host, may be NULL),
 * the state every checkpoint_every steps, and the K - 1 inner states of the
 * last segment (device memory: about ceil(n_steps / K) + 3K states,
 * K = checkpoint_every; K = 1 keeps every state and swe_grad then recomputes
 * nothing). The state is
 * left at step n_steps. Synchronises. Returns SWE_ENAN / SWE_EDRY if a step
 * fails (no tape is made). The tape holds the mesh (not the state). */
swe_status swe_grad_record(swe_state* state, int64_t n_steps, int64_t checkpoint_every,
                           const int32_t* gauge_cells, int32_t n_gauges, double* gauge_h,
                           swe_tape** out);

/* Reverse sweep over the recorded steps. Seeds (host, caller order, any may
 * be NULL = zero): g_h, g_hu, g_hv = dL/d(h, hu, hv) of the final state
 * [n_tris each]; g_gauge = dL/d gauge_h [n_steps * n_gauges]. Outputs (host,
 * caller order, any may be NULL): dL/dh, dL/dhu, dL/dhv of the initial state,
 * dL/dz, dL/dn (n >= 0 assumed). Recomputes each segment of checkpoint_every
 * steps but the last from its checkpoint; returns SWE_ESTATE if a recomputed
 * step did not reproduce the recorded dt. Synchronises. */
swe_status swe_grad(swe_tape* tape, const double* g_h, const double* g_hu, const double* g_hv,
                    const double* g_gauge, double* d_h0, double* d_hu0, double* d_hv0, double* d_z,
                    double* d_n);

/* swe_grad with every seed and output in DEVICE memory (FP64, caller order,
 * the same shapes; any may be NULL as in swe_grad), ordered after the work
 * queued on cuda_stream. Nothing goes through host memory. Synchronises. */
swe_status swe_grad_device(swe_tape* tape, const double* g_h, const double* g_hu,
                           const double* g_hv, const double* g_gauge, double* d_h0,
                           double* d_hu0, double* d_hv0, double* d_z, double* d_n,
                           void* cuda_stream);

/* Copies the gauge depths the tape recorded ([n_steps * n_gauges] FP64,
 * gauge_h[k * n_gauges + j] after step k, as swe_grad_record gives them) to
 * the DEVICE array gauge_h, ordered after the work queued on cuda_stream.
 * Synchronises. */
swe_status swe_tape_gauges_device(const swe_tape* tape, double* gauge_h, void* cuda_stream);

/* info[0] = steps, info[1] = checkpoint interval, info[2] = device time of
 * the recorded forward steps (ms, CUDA events), info[3] = device time of the
 * last swe_grad's recompute and adjoint steps (ms), info[4] = tape bytes. */
swe_status swe_tape_info(const swe_tape* tape, double* info);

void swe_tape_destroy(swe_tape* tape);

/* ---------------------------------------------------------------------------
 * Allocation-free step (no counterpart in the paper).
 *
 * For callers that cannot call cudaMalloc: programs that must not allocate
 * once they are running (fixed memory budgets, real-time loops), and hosts
 * whose device memory comes from their own pool, which a foreign cudaMalloc
 * would bypass. swe_step_edges_static makes one FP64 step of the two-launch
 * kernels (per-edge face outputs, then each cell gathers its three faces)
 * with every input and output a caller-owned device pointer, and its scratch
 * (per-edge face outputs, per-block partial sums, the control word) in one
 * static device array of SWE_STATIC_SCRATCH_BYTES that each GPU loading the
 * library keeps until the process exits. It calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 * Meshes up to SWE_STATIC_MAX_EDGES edges; larger ones (or n_cells > n_edges,
 * which no triangle mesh has) return SWE_EINVAL before any GPU work.
 * The first call on a device looks up the array's device address and the
 * launch sizes (with that device current); make that first call before any
 * stream capture. Calls share the array: each resets what must start at zero,
 * but calls whose work overlaps on the GPU race with each other.
 * --------------------------------------------------------------------------- */
#define SWE_STATIC_SCRATCH_BYTES (16 * 1024 * 1024)
#define SWE_STATIC_MAX_EDGES 417792 /* (16 MiB - 64 KiB) / (5 values * 8 bytes) */

/* Device inputs (caller cell order, FP64 unless noted):
 *   edge_left, edge_right  [n_edges] int32 cells on each side of each edge;
 *                          edge_right = -1 for a wall edge.
 *   edge_nx, edge_ny       [n_edges] unit normal pointing out of edge_left.
 *   edge_len               [n_edges] edge length.
 *   cell_face              [3*n_cells] int32, cell i's face k at [k*n_cells + i]:
 *                          the edge id, with bit 31 set when cell i is that
 *                          edge's right side; face k joins the cell's
 *                          counter-clockwise nodes k and k+1 (faces are summed
 *                          in this order).
 *   cell_area, cell_perim_over_area, gn2 (= g n^2), z, h, hu, hv  [n_cells].
 * Device outputs: h_out, hu_out, hv_out [n_cells] (must not alias the inputs).
 * Host outputs (either may be NULL): *next_dt = CFL dt of the new state,
 * *mass = sum of area * h_out. If either is given the call synchronises the
 * stream and also reports SWE_ENAN / SWE_EDRY; if both are NULL it returns
 * after queueing the work and reports no numerical error (a NaN or an
 * all-dry state is then seen only in the outputs, and the next call resets
 * the control word that recorded it). dt is the length of this step: finite
 * and >= 0, else SWE_EINVAL. Returns SWE_ECUDA if one of its own launches
 * fails; a CUDA error left pending by earlier work is not consumed. */
swe_status swe_step_edges_static(int64_t n_cells, int64_t n_edges, const int32_t* edge_left,
                                 const int32_t* edge_right, const double* edge_nx,
                                 const double* edge_ny, const double* edge_len,
                                 const int32_t* cell_face, const double* cell_area,
                                 const double* cell_perim_over_area, const double* gn2,
                                 const double* z, const double* h, const double* hu,
                                 const double* hv, double g, double courant, double h_eps,
                                 double dt, double* h_out, double* hu_out, double* hv_out,
                                 double* next_dt, double* mass, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Domain decomposition: one mesh split into sub-domains, for one step per
 * sub-domain on its own GPU (or several on one) with a halo exchange and a
 * global time step between steps. The paper names several GPUs on one mesh
 * as future work (Sec. 5); the step itself is Sec. 2.2's.
 *
 * swe_partition_create orders the cells by the Morton code of their
 * centroids and cuts that order into n_parts contiguous ranges of (nearly)
 * equal size. Part p's local mesh holds its own cells plus one ring of
 * ghost cells (cells of other parts sharing an edge with one of its cells),
 * in ascending global order, each triangle with its global node order: every
 * face of an owned cell is then oriented, and every cell's faces ordered, as
 * in the whole mesh, so a step of the local mesh (swe_mesh_create_part)
 * updates the owned cells bit for bit as the whole mesh's step does, when
 * the ghosts hold their owners' current values and the step's dt is the
 * global one. Per step: swe_run(state, 1) on every part; for every ordered
 * pair (from, to), swe_state_halo_pack on `from` with the from-side list of
 * swe_partition_exchange, move the buffer, swe_state_halo_unpack on `to`
 * with the to-side list; swe_state_dt_device on every part, a min over the
 * parts' values (NCCL all-reduce on several GPUs), swe_state_set_dt_min_device
 * on every part. The mass of the whole mesh is the FP64 sum of the parts'
 * swe_copy_out masses (ghosts excluded).
 * --------------------------------------------------------------------------- */
typedef struct swe_partition swe_partition;

/* Builds the partition of a mesh (host arrays as for swe_mesh_create) into
 * n_parts (1 <= n_parts <= n_tris) sub-domains. Host only; copies nothing
 * it keeps but the plan. SWE_EMESH for an invalid mesh. */
swe_status swe_partition_create(const double* xy, int64_t n_nodes, const int32_t* tri,
                                int64_t n_tris, int32_t n_parts, swe_partition** out);

/* sizes[0] = local cells of part `part` (owned and ghost), sizes[1] = ghost
 * cells among them, sizes[2] = local nodes. */
swe_status swe_partition_sizes(const swe_partition* plan, int32_t part, int64_t* sizes);

/* Part `part`'s local mesh, into caller arrays sized by swe_partition_sizes
 * (any may be NULL): cells [local cells] = global cell index of each local
 * cell (ascending), ghost [local cells] = 1 for a ghost cell, else 0,
 * local_xy [2 * local nodes] = coordinates of the local nodes taken from xy
 * (the whole mesh's node array; needed only with local_xy), local_tri
 * [3 * local cells] = local node ids of each local triangle. */
swe_status swe_partition_local_mesh(const swe_partition* plan, int32_t part, const double* xy,
                                    int32_t* cells, uint8_t* ghost, double* local_xy,
                                    int32_t* local_tri);

/* The cells owned by part `from` that part `to` holds as ghosts, in
 * ascending global order: *n of them; from_cells[k] = its local index in
 * `from`, to_cells[k] = its local index in `to` (either may be NULL: call
 * once with both NULL to size them). from == to gives *n = 0. */
swe_status swe_partition_exchange(const swe_partition* plan, int32_t from, int32_t to, int64_t* n,
                                  int32_t* from_cells, int32_t* to_cells);

void swe_partition_destroy(swe_partition* plan);

/* swe_mesh_create for a sub-domain's local mesh: ghost [n_tris] (host,
 * caller order) marks the ghost cells, which take part in the faces of the
 * owned cells but not in the CFL time step nor in the mass integral (their
 * own updates are overwritten by the halo exchange). Needs SWE_KERNEL_TILED
 * (or AUTO), else SWE_EINVAL. */
swe_status swe_mesh_create_part(const double* xy, int64_t n_nodes, const int32_t* tri,
                                int64_t n_tris, const uint8_t* ghost, const swe_params* params,
                                void* cuda_stream, swe_mesh** out);

/* Queues, on the mesh's stream, buf[3 k + f] = field f (h, hu, hv; FP64) of
 * local cell cells[k] of the current state, k < n. cells and buf are DEVICE
 * arrays; entries outside [0, n_tris) are skipped. SWE_ESTATE unless the
 * mesh came from swe_mesh_create_part. No synchronisation. */
swe_status swe_state_halo_pack(const swe_state* state, const int32_t* cells, int64_t n,
                               double* buf);

/* Queues the reverse: field f of local cell cells[k] of the current state =
 * buf[3 k + f] (DEVICE arrays), k < n. No synchronisation. */
swe_status swe_state_halo_unpack(swe_state* state, const int32_t* cells, int64_t n,
                                 const double* buf);

/* Queues a copy of the CFL time step of the current state (Sec. 2.2,
 * Courant 0.7, over its non-ghost cells) to the DEVICE double *dt.
 * Single-scenario meshes. No synchronisation. */
swe_status swe_state_dt_device(const swe_state* state, double* dt);

/* Queues: the next step uses the smallest of the n DEVICE doubles dts[0..n)
 * as its time step (the global CFL step of a decomposed mesh). Makes the
 * state open-ended (no end time). Single-scenario meshes. No
 * synchronisation. */
swe_status swe_state_set_dt_min_device(swe_state* state, const double* dts, int32_t n);

/* Measurement helper (no counterpart in the paper): FP64 fused multiply-add
 * throughput of the current device, for the FP64 path's arithmetic roofline.
 * Runs a kernel of independent DFMA chains on every SM on `cuda_stream`
 * (NULL: the default stream), timed with CUDA events; *tflops = FP64 flops
 * (2 per fused multiply-add) per second / 1e12. Allocates a small output
 * buffer, synchronises the stream. SWE_ECUDA on a CUDA error. */
swe_status swe_fp64_fma_rate(void* cuda_stream, double* tflops);

/* Static description of a status code. */
const char* swe_strerror(swe_status status);

/* Message of the last CUDA runtime error seen by this thread ("" if none). */
const char* swe_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SWE_H */

/*
 * lbibm.h - C ABI of the GB300 lattice-Boltzmann + immersed-boundary library.
 *
 * The library advances the blood-flow model of Gusenbauer et al., "A tunable
 * cancer cell filter using magnetic beads: cellular and fluid dynamic
 * simulations" (arXiv:1110.0995) on one NVIDIA GB300 (sm_103a):
 *
 *   - D3Q19 lattice-Boltzmann with an external force term (Sec. 2.1),
 *   - bounce-back walls and fixed obstacle nodes such as bead chains and
 *     microposts (Sec. 2.4, 2.5),
 *   - the immersed-boundary cycle (Sec. 2.2): velocity transmitted from the
 *     grid to the IB points, node forces from the cell membranes (Sec. 2.3.1:
 *     stretching K^S, bending K^B, local/global area K^A_l/K^A_g, volume K^V),
 *     forces spread back onto the grid, fluid and points advanced.
 *
 * Conventions (all entry points):
 *   - Lattice units.  Lattice node (x, y, z), 0 <= x < nx etc., has linear
 *     index p = x + nx * (y + ny * z).  Non-periodic axes carry halfway
 *     bounce-back walls at -1/2 and n - 1/2.
 *   - The caller owns every array it passes.  Inputs are copied during the
 *     call; outputs are written into caller buffers, on the host unless a
 *     `dst_is_device` argument says the pointer is device memory (for example
 *     a torch tensor's data pointer on the context's device).
 *   - The library owns all device memory of a context (allocated in
 *     lb_create / ibm_add_mesh / lb_set_obstacles, freed in lb_destroy).
 *   - Work is queued on the CUDA stream given to lb_create (NULL = the legacy
 *     default stream).  Calls that return data synchronise that stream.
 *   - No exception or abort crosses the ABI.  Every call returns an
 *     lb_status; lb_last_error(ctx) gives a message (lb_last_error(NULL) for
 *     the calls that have no context).  A CUDA error poisons the
 *     context: every later call returns LB_ERR_CUDA.
 *   - One context per stream; calls on one context are not thread-safe.
 */
#ifndef LBIBM_H
#define LBIBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_ctx lb_ctx;

typedef enum {
    LB_OK = 0,
    LB_ERR_ARG = 1,      /* invalid argument (sizes, tau <= 1/2, open mesh, ...) */
    LB_ERR_STATE = 2,    /* call not allowed in the context's current state */
    LB_ERR_CUDA = 3,     /* CUDA runtime error; the context is poisoned */
    LB_ERR_OOM = 4,      /* device allocation failed */
    LB_ERR_NUMERIC = 5,  /* non-finite value or |u| above the stability bound */
    LB_ERR_TIMEOUT = 6   /* a bounded device-side wait ran out */
} lb_status;

/* Storage of the populations.  Arithmetic is FP32 in every mode.
 * LB_F32:          shifted populations h_i = f_i - w_i (rho0 = 1) in FP32.
 * LB_F16_SHIFTED:  h_i / w_i stored as IEEE binary16.
 * LB_BF16_SHIFTED: h_i / w_i stored as bfloat16.
 * 16-bit stores round stochastically: up with probability equal to the
 * discarded fraction, the random bits a hash of the node index and the bit
 * patterns of its moments (unbiased per store, independent between nodes,
 * reproducible run to run).  Rounding to nearest would give a region of
 * near-uniform flow one coherent error per step that viscosity does not damp. */
typedef enum { LB_F32 = 0, LB_F16_SHIFTED = 1, LB_BF16_SHIFTED = 2 } lb_storage;

typedef struct {
    int nx, ny, nz;              /* lattice dimensions, each >= 1; nx*ny*nz <= 2^31 - 1 */
    double tau;                  /* BGK relaxation time (Sec. 2.1), > 1/2 */
    double body_force[3];        /* uniform force density at every fluid node (finite) */
    int periodic[3];             /* 1 = periodic axis, 0 = bounce-back walls */
    double wall_velocity[2][3];  /* velocity of the y = -1/2 and y = ny - 1/2 walls (finite) */
    lb_storage storage;
    int reserved[4];             /* must be zero */
} lb_params;

/* Membrane moduli of one cell (Sec. 2.3.1, Table 1). */
typedef struct {
    double ks;   /* stretching K^S (neo-Hookean bond) */
    double kb;   /* bending K^B (dihedral angle) */
    double kal;  /* local area K^A_l (per triangle) */
    double kag;  /* global area K^A_g (whole cell) */
    double kv;   /* volume K^V */
} ibm_moduli;

/* Create a context: allocates the lattice (two population buffers, force and
 * velocity fields) and fills it with the rest equilibrium rho = 1, u = 0.
 * `cuda_stream` is a cudaStream_t (or NULL).  LB_ERR_ARG for invalid params
 * (checked on the host before any CUDA call), LB_ERR_OOM if the lattice does
 * not fit. */
lb_status lb_create(const lb_params* params, void* cuda_stream, lb_ctx** out);

/* Batched variant: `n_channels` independent lattices (one params entry each,
 * all with the same storage) advanced together, one launch per kernel per
 * step for the whole batch (Sec. 3.1's gap sweep is such a batch).  Channel
 * k's meshes and obstacles are addressed with lb_select_channel. */
lb_status lb_create_batch(const lb_params* params, int n_channels, void* cuda_stream, lb_ctx** out);

/* Select the channel that later lb_set_obstacles / ibm_add_mesh /
 * lb_get_fields / lb_get_populations calls refer to (default 0). */
lb_status lb_select_channel(lb_ctx* ctx, int channel);

/* Free all device memory of the context.  NULL is accepted. */
lb_status lb_destroy(lb_ctx* ctx);

/* Collisions between cells and with walls and beads (Sec. 2.4: a soft
 * potential between mesh nodes of different cells and between cells and
 * walls, cut at an interaction radius; form and constants not printed).
 * Reading: harmonic soft sphere, a force k (dc - d) along the separation for
 * d < dc, between nodes of different cells of a channel (x minimum image when
 * x is periodic), between a node and the surface of a bead of
 * lb_set_obstacles (d = |x - c| - r), and between a node and a wall of a
 * non-periodic axis (walls half a link outside the first and last node),
 * added to the membrane forces before spreading.  k = 0 (the default) turns
 * it off.  Before the first step; not with the differentiable variant
 * (LB_ERR_STATE).  Candidate lists hold 32 neighbour cells and 256 beads per
 * cell; an overflow is reported by lb_diagnostics (LB_ERR_STATE). */
lb_status lb_set_repulsion(lb_ctx* ctx, double k, double dc);

/* IB points with mass (Sec. 2.2: m d^2X/dt^2 = F; the coupling force comes
 * from the motion of a point relative to the fluid).  Reading: a frictional
 * coupling -gamma (V - U), U the fluid velocity of the last collision
 * interpolated at X; the membrane and collision forces F act on the points
 * only.  Each cycle: kick V = W + F / mass, then the drift under the drag with
 * U held, solved exactly (a = gamma / mass, p1 = (1 - e^-a) / a):
 * X += U + p1 (V - U), W = U + e^-a (V - U); the fluid receives the drag's
 * impulse gamma p1 (V - U), spread at the old position.  W (the point
 * velocity after the drift) starts at zero.  mass = 0 (the default): massless
 * points advected with the interpolated velocity.  mass > 0, gamma >= 0,
 * finite; before the first step (LB_ERR_STATE); not with the differentiable
 * variant or lb_adjoint.  Uses the sequential schedule. */
lb_status lb_set_ib_dynamics(lb_ctx* ctx, double mass, double gamma);

/* Deterministic cycle (on = 1): the spreading kernel accumulates the force
 * density in 64-bit fixed point (2^-40; integer sums do not depend on the
 * order of the atomic additions) and a conversion kernel writes it to the
 * FP32 force field, so that repeated runs give bit-identical populations and
 * positions (one more kernel per cycle, 24 bytes per lattice node).  on = 0
 * (the default): FP32 atomic additions, whose order varies from run to run at
 * the rounding level.  Not with collisions (LB_ERR_STATE); the adjoint keeps
 * FP32 atomics.  Uses the sequential schedule. */
lb_status lb_set_deterministic(lb_ctx* ctx, int on);

/* Velocities W of one mesh's points (n x 3, host) after the last step
 * (zeros for massless points). */
lb_status ibm_get_velocities(lb_ctx* ctx, int mesh_id, double* v);

/* Differentiable variant (gradient of a filter objective; single-channel
 * contexts, before the first step).  The beads become a smooth solid
 * fraction phi(x) = 1 - prod_k (1 - phi_k(x)),
 * phi_k = 1/2 [1 - tanh((|x - c_k| - r_k) / delta)], entering every collision
 * as the implicit Brinkman force -alpha phi rho u:
 * u = (sum_i f_i e_i + g/2) / (rho (1 + alpha phi / 2)) and the Guo source
 * takes g - alpha phi rho u.  The paper's beads are bounce-back nodes
 * (Sec. 2.4, 2.5), whose mask is piecewise constant in a bead centre; this
 * smooth form makes the objective differentiable.  beads: n x {cx, cy, cz, r}
 * (host, copied).  Walls stay bounce-back; lb_set_obstacles masks, if any,
 * still apply.  Selects the one-node-per-thread stream-collide variant.
 * LB_ERR_STATE after the first step, LB_ERR_ARG for bad data. */
lb_status lb_set_brinkman(lb_ctx* ctx, const double* beads, int n, double alpha, double delta);

/* Gradient of the filter objective J = (mean x of the objective mesh's nodes
 * after n_steps cycles) - (the same now), for the differentiable variant
 * (lb_set_brinkman; FP32 populations, one channel), by the discrete adjoint
 * of the cycle: n_steps forward cycles keeping the state every ckpt_every
 * cycles, then per segment a recompute that keeps each cycle's data and the
 * reverse sweep through it (interpolation, stream-collide with the Brinkman
 * term, spreading, membrane forces).  Outputs (host, caller-owned): *J;
 * grad_beads[3 k + axis] = dJ/d(centre of bead k), n_beads x 3; *grad_ks and
 * *grad_kb = dJ/d(ks), dJ/d(kb) of the objective mesh's cell.  Any output may
 * be NULL.  Afterwards the context holds the state after the n_steps cycles,
 * as lb_step(n_steps) leaves it.  Device workspace: about
 * (n_steps / ckpt_every + ckpt_every) x (19 x 4 B) x nodes, kept for the next
 * call of the same shape.  LB_ERR_STATE without lb_set_brinkman or with
 * per-kernel timing on; LB_ERR_OOM if the workspace does not fit. */
lb_status lb_adjoint(lb_ctx* ctx, int n_steps, int ckpt_every, int objective_mesh, double* J, double* grad_beads,
                     double* grad_ks, double* grad_kb);

/* Obstacles (Sec. 2.4, 2.5): every lattice node inside or on one of the `n`
 * spheres spheres[4k..4k+3] = (cx, cy, cz, r) becomes a solid bounce-back
 * node; the test |x - c|^2 <= r^2 is evaluated in double from the float
 * inputs.  `extra_mask` (optional, nx*ny*nz bytes, nonzero = solid) adds
 * arbitrary solid nodes.  Replaces any previous obstacles.  Only before the
 * first lb_step (LB_ERR_STATE otherwise). */
lb_status lb_set_obstacles(lb_ctx* ctx, const float* spheres, int n, const uint8_t* extra_mask);

/* Obstacle map of the selected channel: N bytes, 1 = solid node (host). */
lb_status lb_get_mask(lb_ctx* ctx, uint8_t* solid);

/* Add one closed cell membrane (Sec. 2.2, 2.3): `rest_xyz` (n_nodes x 3,
 * lattice units) is the rest shape already placed in the channel and also the
 * initial position; `tris` (n_tris x 3) are outward counter-clockwise
 * triangles.  The mesh must be a closed oriented 2-manifold with positive
 * volume and node valence <= 64 (LB_ERR_ARG otherwise). Positions are kept
 * in 64-bit fixed point with 2^-40 lu resolution.  Only before the first
 * lb_step.  *mesh_id receives the index of the mesh within the channel.
 * Meshes with the same triangle list share one connectivity check; the
 * element tables are built by the first lb_step. */
lb_status ibm_add_mesh(lb_ctx* ctx, const double* rest_xyz, int n_nodes, const int32_t* tris, int n_tris,
                       const ibm_moduli* moduli, int* mesh_id);

/* The check ibm_add_mesh applies to a cell membrane mesh (Sec. 2.3.1: a
 * closed triangulated surface of IB points), without a context and without
 * the GPU (host code only): n_nodes >= 4 and n_tris >= 4, finite
 * positions with |x| < 4e6, indices in range, no degenerate triangle, every
 * directed edge in exactly one triangle and its reverse in another (closed,
 * consistently oriented), every node a single fan of at most 64 triangles,
 * no isolated node, positive volume (outward orientation).  Returns LB_OK or
 * LB_ERR_ARG; when `why` is not NULL the reason (empty when LB_OK) is
 * written into it, at most why_len - 1 characters and a terminating NUL. */
lb_status ibm_check_mesh(const double* rest_xyz, int n_nodes, const int32_t* tris, int n_tris, char* why,
                         int why_len);

/* Overwrite the current node positions of one mesh (n_nodes x 3, host). */
lb_status ibm_set_nodes(lb_ctx* ctx, int mesh_id, const double* xyz);

/* Advance `n_steps` immersed-boundary cycles (Sec. 2.2): per-cell area and
 * volume (FP64 reduction), node forces, spreading, fused stream-collide with
 * force, velocity interpolation and point advance.  Asynchronous on the
 * context's stream; launched as a CUDA graph after the first call. */
lb_status lb_step(lb_ctx* ctx, int n_steps);

/* Variant of the fused stream-collide kernel.  nodes_per_thread 1, 2 or 4:
 * consecutive x-nodes per thread (every channel's nx a multiple of it), with
 * block_size 128 or 256; with 2 the pair's moments and collision run as packed
 * two-lane FP32 operations.  nodes_per_thread 0: staged variant (rows copied to
 * shared memory asynchronously; block_size 256; every channel's row of nx
 * populations a multiple of 16 bytes and nx <= 512).  nodes_per_thread -1:
 * pipelined variant (persistent warps, block_size 128 or 256).
 * nodes_per_thread -2: TMA-staged variant (tensor copies of every direction's
 * source rows into shared memory, double-buffered, one node per thread;
 * block_size 256 or 512 = nodes per tile); FP32 storage, one channel, walls
 * (not periodic) in y and z, nx in {32, 64, 128, 256} dividing block_size and
 * ny a multiple of block_size / nx.  A block that gives up waiting for its
 * copies makes lb_diagnostics return LB_ERR_TIMEOUT.  The default is 1 node per
 * thread, 128 threads, for FP32 storage, and for 16-bit storage 4 nodes per
 * thread, 64 threads where every nx is a multiple of 4 (the 16-bit variant
 * with 4 nodes per thread keeps each direction's four values packed in one
 * 64-bit word until the node pairs are unpacked in turn).  LB_ERR_ARG for an unsupported pair.  Results depend
 * on the variant only through FP32 rounding (the two-node variant orders the
 * collision's operations differently). */
lb_status lb_set_kernel_config(lb_ctx* ctx, int nodes_per_thread, int block_size);
lb_status lb_get_kernel_config(lb_ctx* ctx, int* nodes_per_thread, int* block_size);

/* L2 prefetch distance of the fused stream-collide kernel (one, two or four
 * nodes per thread), in lattice nodes: each block asks L2 for the source
 * populations (every direction's plane) of the nodes nodes_ahead past its
 * own, so that blocks running later find their pulls in L2 rather than in
 * HBM.  A performance setting only (Sec. 2.1's update is unchanged; results
 * are bit-identical for every distance).  0 = off (the default); otherwise a
 * multiple of 256 up to 2^24, else LB_ERR_ARG.  The bound on the useful
 * distance is the L2 (19 x 4 bytes per node of distance for FP32 storage). */
lb_status lb_set_prefetch(lb_ctx* ctx, int nodes_ahead);
lb_status lb_get_prefetch(lb_ctx* ctx, int* nodes_ahead);

/* Step schedule.  overlapped = 0 (default): the four kernels of the cycle
 * run one after another, each launched as a programmatic dependent of its
 * predecessor (its blocks are scheduled during the predecessor's last wave
 * and wait for the predecessor to complete before touching memory).
 * overlapped = 2: the same cycle with ordinary launches.  overlapped = 1: when
 * the context has IB meshes, the stream-collide variant has one node per
 * thread and none of collisions, points with mass, the deterministic cycle
 * or the differentiable variant is on (otherwise the sequential cycle with
 * programmatic dependent launches runs), each cycle runs the immersed-boundary kernels on a second,
 * higher-priority stream concurrently with the stream-collide of every
 * 32-node group that no IB point can reach in that step, then updates the
 * reachable groups; the results equal the sequential cycle as long as no IB
 * point moves one lattice unit or more in one step (a spreading target
 * outside the reachable set is counted and reported by lb_diagnostics as
 * LB_ERR_NUMERIC).  On GB300 the overlapped schedule is currently slower: the
 * latency-bound IB kernels hold SM slots that the concurrent stream-collide
 * needs.  Per-kernel timing (lb_set_timing) always uses the sequential
 * schedule with ordinary launches.  All schedules give the same results.
 * lb_get_schedule reports the schedule the next lb_step will use. */
lb_status lb_set_schedule(lb_ctx* ctx, int overlapped);
lb_status lb_get_schedule(lb_ctx* ctx, int* overlapped);

/* Autotuner: times every supported stream-collide variant on this context's
 * lattice (`repeats` launches each, CUDA events), selects the fastest, then
 * times its L2 prefetch distances (0, 65536, 131072, 262144 nodes; variants
 * with 1, 2 or 4 nodes per thread) and keeps the fastest (lb_get_prefetch
 * reads it), and returns the variant with its mean time per launch in ms.
 * Only before the first lb_step (LB_ERR_STATE otherwise): there, repeated
 * launches leave the state unchanged. */
lb_status lb_autotune(lb_ctx* ctx, int repeats, int* nodes_per_thread, int* block_size, double* ms);

/* Wait for the context's stream and report any pending error. */
lb_status lb_synchronize(lb_ctx* ctx);

/* Density (N floats) and velocity (3 x N floats, SoA: u[d*N + p]) of the last
 * step's collision, for the selected channel; either pointer may be NULL.
 * The velocity is the force-corrected u = (sum_i f_i e_i + g/2) / rho; solid
 * nodes report rho = 1, u = 0.  Before any step: rho = 1, u = 0. */
lb_status lb_get_fields(lb_ctx* ctx, float* rho, float* u, int dst_is_device);

/* Pre-collision populations f_i(x, t) of the next step (19 x N doubles,
 * direction-major f[i*N + p], D3Q19 order: rest, +-x, +-y, +-z, then
 * (+-1,+-1,0), (+-1,0,+-1), (0,+-1,+-1) with opposite directions adjacent),
 * for the selected channel, on the host. */
lb_status lb_get_populations(lb_ctx* ctx, double* f);

/* Set the pre-collision populations of the next step (same layout). */
lb_status lb_set_populations(lb_ctx* ctx, const double* f);

/* Current node positions of one mesh of the selected channel (n x 3, host). */
lb_status ibm_get_nodes(lb_ctx* ctx, int mesh_id, double* xyz);

/* Current positions of every mesh of the selected channel, in the order the
 * meshes were added, concatenated into xyz (sum of their node counts x 3,
 * host, caller-owned).  One device-to-host transfer per run of adjacent meshes
 * through a page-locked staging buffer, one wait.  The paper's filter runs
 * record cell trajectories (Sec. 3); this is that readback. */
lb_status ibm_get_all_nodes(lb_ctx* ctx, double* xyz);

/* Asynchronous form of ibm_get_all_nodes for trajectory recording alongside
 * the stepping: enqueues on the context's stream the conversion of the
 * selected channel's positions to double (on the device) and their copy into
 * xyz (host, caller-owned, page-locked for the copy to overlap later steps),
 * then returns.  slot (0 or 1) names the readback; xyz is complete once
 * lb_readback_wait(ctx, slot) has returned LB_OK, and must not be reused
 * before.  Alternating slots lets the host consume one readback while the
 * next runs behind further steps. */
lb_status ibm_get_all_nodes_async(lb_ctx* ctx, double* xyz, int slot);
lb_status lb_readback_wait(lb_ctx* ctx, int slot);

/* Node forces spread in the last step (n x 3, host). */
lb_status ibm_get_forces(lb_ctx* ctx, int mesh_id, double* f);

/* Per-cell surface area and volume at the current positions (the rest values
 * plus the sums of the per-triangle changes, added exactly in 2^-40 fixed
 * point; FP64 results), for every mesh of the selected channel, in mesh order
 * (host). */
lb_status ibm_get_area_volume(lb_ctx* ctx, double* area, double* volume);

/* Surface area and enclosed volume of closed triangle meshes, allocating no
 * device memory.  The paper has no counterpart to this entry point: it serves
 * callers that cannot allocate device memory (code under a framework that
 * owns the whole device memory pool, latency-critical loops that cannot
 * afford cudaMalloc's implicit synchronisation, embedded callers with a fixed
 * memory budget).  It computes what ibm_get_area_volume reports, from caller
 * buffers instead of a context:
 *   xyz             device, n_nodes x 3 doubles (node positions)
 *   tris            device, n_tris x 3 int32 node indices, outward counter-clockwise
 *   cell_tri_start  device, n_cells + 1 int32: cell c owns triangles
 *                   [cell_tri_start[c], cell_tri_start[c+1])
 *   cell_tri_start_host  the same offsets in host memory (sizes the grid;
 *                   offsets on the device that disagree with these give
 *                   wrong sums but no access outside the scratch array)
 *   area, volume    device, n_cells doubles each (outputs)
 * FP64 throughout; queued on cuda_stream (NULL = legacy default stream),
 * asynchronous.  Scratch is a fixed 1 MiB device array (65,536 partial sums
 * of 256 triangles each) that every GPU loading the library holds until the
 * process exits: LB_ERR_ARG when n_cells times the largest number of
 * 256-triangle chunks of one cell exceeds 65,536, or n_cells > 65,535.  The
 * first call on a device looks the array's address up (cudaGetSymbolAddress)
 * and so does the first call after the device's current context changed (a
 * cudaDeviceReset, or another driver context made current); make such a call
 * before any stream capture.  Every call shares the array, so calls that
 * overlap on the GPU race.  LB_ERR_CUDA when a launch is refused; an error
 * left over from an earlier, unrelated call is not consumed.  Calls no
 * cudaMalloc or cudaFree.  n_cells = 0 does nothing and returns LB_OK. */
lb_status ibm_area_volume_noalloc(const double* xyz, const int32_t* tris, const int32_t* cell_tri_start,
                                  const int32_t* cell_tri_start_host, int n_cells, double* area, double* volume,
                                  void* cuda_stream);

/* ---- magnetic bead assembly (Sec. 2.5), context-free ----
 * The force of bead a on bead b with moments m_a, m_b at r = x_b - x_a is the
 * printed dipole interaction (its bracket closed after the last term),
 *   F = 3c / |r|^5 [(m_a.r) m_b + (m_b.r) m_a + (m_a.m_b) r - 5 (m_a.r)(m_b.r) r / |r|^2],
 * c = mu0 / (4 pi) in the caller's units, plus for |r| < 2R a contact force
 * k (2R - |r|) along r (the paper adds collision forces without a form;
 * reading: harmonic).  Separations use the minimum image on periodic axes.
 * The external field's gradient force needs the charge-sheet field, which
 * the paper does not give: moments are inputs (e.g. all along a uniform
 * field).  FP32 on the device, all pairs. */
typedef struct {
    double mu0_4pi;      /* c */
    double radius;       /* R >= 0 */
    double k_contact;    /* k >= 0 */
    double mobility;     /* overdamped friction: velocity per unit force */
    double dt;           /* time step of bead_relax */
    double box[3];       /* box edges; > 0 on periodic axes */
    int periodic[3];
    int reserved[5];     /* must be zero */
} bead_params;

/* Forces on n beads (xyz, moments: n x 3 host arrays; F: n x 3 host output).
 * Coincident beads are undefined.  LB_ERR_ARG for n < 1, null pointers or bad
 * parameters; LB_ERR_OOM / LB_ERR_CUDA on device failure.  Synchronous on
 * `cuda_stream` (NULL = default stream); allocates its device buffers. */
lb_status bead_forces(const double* xyz, const double* moments, int n, const bead_params* p, double* F,
                      void* cuda_stream);

/* Overdamped bead motion: `steps` steps of x += mobility * F(x) * dt, every
 * bead from the positions of the same step, wrapped into the box on periodic
 * axes; xyz (n x 3, host) is updated in place.  Errors as bead_forces. */
lb_status bead_relax(double* xyz, const double* moments, int n, const bead_params* p, int steps, void* cuda_stream);

/* Conservation diagnostics of the selected channel, FP64 on the device:
 * out[0] = sum of rho over fluid nodes, out[1..3] = sum of sum_i e_i f_i
 * after the last collision, out[4] = number of non-finite populations,
 * out[5] = max |u| over fluid nodes.  Returns LB_ERR_NUMERIC when out[4] > 0
 * or out[5] > `u_max` (pass u_max <= 0 to skip the bound), or when an IB
 * point moved a lattice unit in one step under the overlapped schedule;
 * LB_ERR_STATE when the collision candidate lists overflowed; LB_ERR_TIMEOUT
 * when a block of the TMA-staged variant gave up waiting for its copies.  The
 * sums are filled in every case. */
lb_status lb_diagnostics(lb_ctx* ctx, double u_max, double out[6]);

/* Number of completed steps. */
lb_status lb_get_step(lb_ctx* ctx, int64_t* step);

/* Checkpoint: with buf == NULL, *bytes receives the size; otherwise the
 * whole device state (populations, force fields, positions, step; for IB
 * points with mass also their velocities and the fluid velocity of the last
 * collision) is copied into buf (host, *bytes large enough). */
lb_status lb_save_state(lb_ctx* ctx, void* buf, size_t* bytes);
lb_status lb_load_state(lb_ctx* ctx, const void* buf, size_t bytes);

/* Optional per-kernel timing.  Kernel classes: 0 = element pass (cell area /
 * volume sums and element forces),
 * 1 = membrane forces + spreading, 2 = fused stream-collide,
 * 3 = interpolation + advance.  With kernel_mask != 0 (bit k for class k,
 * 15 = all) lb_step launches the kernels one by one (no graph) and records a
 * pair of CUDA events on the context's stream around every launch of a
 * selected class; 0 returns to graph launches.  LB_ERR_ARG outside 0..15.
 * lb_kernel_times synchronises the stream and returns, per class, the
 * accumulated event milliseconds (0 for classes not timed) and the number of
 * launches enqueued (timed or not) since the previous call, then resets both. */
lb_status lb_set_timing(lb_ctx* ctx, int kernel_mask);
lb_status lb_kernel_times(lb_ctx* ctx, double ms[4], int64_t launches[4]);

/* Message of the last error on this context (never NULL; valid until the
 * context's next failing call).  With ctx == NULL: the message of the last
 * failed call of the calling thread that has no context (lb_create,
 * lb_create_batch, ibm_check_mesh, bead_forces, bead_relax), "no error"
 * before any; valid until that thread's next such failure. */
const char* lb_last_error(const lb_ctx* ctx);

/* Library version: major * 10000 + minor * 100 + patch. */
int lb_version(void);

/* Debugging aid for out-of-bounds device writes (there is no memory checker
 * to run): with bytes > 0, every device allocation of the contexts created
 * afterwards gets `bytes` (rounded up to a multiple of 256) of a fixed byte
 * pattern before and after it; 0 turns it off for later contexts.  Process-
 * wide, host-only; LB_ERR_ARG above 1 GiB.  Not a paper operation. */
lb_status lb_set_guard_zones(size_t bytes);

/* Bytes of the context's guard zones that no longer hold the pattern (0 when
 * no kernel wrote past either end of any of its allocations; 0 as well for a
 * context created without guard zones).  Waits for the context's stream.
 * self_test != 0 first changes one byte of every zone from the host, counts,
 * and restores them: the count is then 2 per allocation plus any damage. */
lb_status lb_check_guard_zones(lb_ctx* ctx, int self_test, int64_t* damaged_bytes);

#ifdef __cplusplus
}
#endif

#endif /* LBIBM_H */

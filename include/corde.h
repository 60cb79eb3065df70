/*
 * corde.h - C ABI of the GB300 (sm_103a) CoRdE Cosserat-rod time stepper.
 *
 * The method is the CoRdE rod of Korzeniowski, Hald and Bello, "Massively-Parallel
 * Implementation of Inextensible Elastic Rods Using Inter-block GPU Synchronization":
 * N centreline points r_i and N-1 material frames stored as unit quaternions q_j
 * (Section 2.1, "Discretization"); stretch energy (Eq. 2), bend/twist energy with the
 * Darboux vector from adjacent quaternions (Eq. 3, 5, 6), the parallel-constraint
 * penalty (Eq. 7-8); per time step the order of Fig. 5: external forces, elastic forces
 * and torques, force integration, j iterations of distance-constraint impulses
 * (inextensible variant, Section 2.1 "Constraints"), then semi-implicit Euler
 * integration of the velocities.  Many time steps run inside one kernel launch
 * (Section 2.2): the paper's launch takes the number of steps, the number of
 * constraint iterations, the material and the haptic input, which map to rod_step,
 * RodParams and rod_set_input.
 *
 * Conventions
 *  - A handle holds a batch of independent rods (a single rod is a batch of one).
 *    Rod r has n_nodes[r] = N_r nodes and N_r - 1 frames.  Elements are numbered
 *    globally: rod r owns elements [off_r, off_r + N_r), off_r = sum of earlier N.
 *    Element i carries node i and, except for a rod's last element, frame i.
 *  - Quaternions are (x, y, z, w) with w the real part; they map body to world, the
 *    frame's third director d3 = R(q) e_z is the tangent direction.
 *  - Angular velocities are in the body frame.
 *  - Node 0 and frame 0 of a rod with clamp != 0 are kinematic (the clamped or
 *    driven base): their velocities come from the drive input, forces do not move them.
 *  - Pointer arguments may point to host memory (pageable or pinned) or device memory
 *    unless stated otherwise; the library copies with cudaMemcpyAsync (default kind).
 *    Caller buffers are borrowed for the duration of the call on the given stream and
 *    are never freed by the library.  `stream` is a cudaStream_t (NULL = legacy default).
 *  - All calls are asynchronous on `stream` unless stated otherwise.  Return value:
 *    CORDE_OK (0) or a negative CORDE_ERR_* code; rod_last_error() gives a message.
 *    Argument errors are detected on the host before anything is enqueued.
 *  - Device state is owned by the handle and freed by rod_destroy.
 */
#ifndef CORDE_H_
#define CORDE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CORDE_OK 0
#define CORDE_ERR_ARG (-1)         /* invalid argument (sizes, NULL, parameter range)  */
#define CORDE_ERR_CUDA (-2)        /* a CUDA runtime call failed                       */
#define CORDE_ERR_OOM (-3)         /* device allocation failed                         */
#define CORDE_ERR_UNSUPPORTED (-4) /* rod longer than any kernel variant, or no GPU    */
#define CORDE_ERR_NONFINITE (-5)   /* diagnostics found a non-finite state             */
#define CORDE_ERR_BUSY (-6)        /* no consistent mailbox snapshot after many tries   */

typedef struct corde_rods* rod_handle;

/* Material, geometry and stepping parameters of one rod (SI units).
 *  length, radius          rod length L and cross-section radius r
 *  E_bend, E_stretch, G    Young's moduli for bending and stretching, shear modulus;
 *                          K1 = K2 = E_bend pi r^4/4, K3 = G pi r^4/2 (Eq. 3, read with
 *                          the second moments), Ks = E_stretch pi r^2 (Eq. 2)
 *  density                 mass density rho; node masses rho pi r^2 l0 (half at ends)
 *  Kp                      penalty constant of Eq. 8 (N); <= 0 selects 100 * 4 K1 / L^2
 *  damping_alpha           mass-proportional internal friction alpha (1/s), implicit
 *  mass_scale, inertia_scale  factors on the inertial node masses and frame inertias
 *                          (gravity keeps the physical mass); <= 0 selects the smallest
 *                          factor that keeps the estimated highest mode at omega dt <= 0.5
 *  dt                      time step (s)
 *  gravity                 acceleration vector (m/s^2)
 *  n_nodes                 N >= 2
 *  n_iters                 constraint iterations per step (Fig. 5 "j"), >= 0
 *  inextensible            1: distance constraints replace Eq. 2; 0: extensible rod
 *  clamp                   1: node 0 and frame 0 are kinematic (driven base); 0: free
 */
typedef struct {
  double length, radius, E_bend, E_stretch, G, density, Kp, damping_alpha;
  double mass_scale, inertia_scale, dt;
  double gravity[3];
  int n_nodes, n_iters, inextensible, clamp;
} RodParams;

/* Create a batch of n_rods rods.
 *  params     [n_rods] host array.
 *  pos        [sum N][3]  initial node positions.
 *  quat       [sum (N-1)][4] initial frames (x, y, z, w), unit norm.
 *  rest_quat  [sum (N-1)][4] rest frames defining the intrinsic Darboux vectors u-hat
 *             of Eq. 3 (computed from them with the same formula as u), or NULL for a
 *             straight, untwisted rest shape (u-hat = 0).
 *  vel        [sum N][3] initial velocities or NULL (zero).
 *  omega      [sum (N-1)][3] initial body angular velocities or NULL (zero).
 *  stiff_mul  [sum (N-2)][3] per-joint multipliers of (K1, K2, K3) or NULL (ones).
 * Frames of one rod must be on one hemisphere (q_j . q_{j+1} > 0).
 * Blocks until the device state is initialised.  On success *out receives the handle. */
int rod_create(int n_rods, const RodParams* params, const float* pos, const float* quat,
               const float* rest_quat, const float* vel, const float* omega,
               const float* stiff_mul, void* stream, rod_handle* out);

/* Advance every rod by n_steps time steps in one persistent launch per kernel variant
 * of the handle's plan (one launch for a single rod).  drive: [n_rods][8] device
 * pointer (v_x v_y v_z beta w_x w_y w_z _), the base velocity and body angular velocity
 * held for the whole call (beta: binding offset of an inner rod, see rod_bind), or NULL
 * to use the values last given to rod_set_input (initially zero).  n_steps >= 0. */
int rod_step(rod_handle h, int n_steps, const float* drive, void* stream);

/* One haptic tick in one call (the haptic loop of Section 2.2: the input goes in, the
 * kernel runs its steps, the state comes out for the host): as rod_step, and the kernels
 * write the positions after the last step to pos_out, [n_elements][4] floats (x, y, z,
 * inverse mass), in their epilogue.  drive and pos_out may be device memory or mapped
 * pinned host memory (cudaHostAlloc: mapped by default under unified addressing); over a
 * coherent CPU-GPU link the kernels then read the drive and write the positions across
 * the link, with no separate copy.  Both must be 16-byte aligned (CORDE_ERR_ARG
 * otherwise).  pos_out NULL: exactly rod_step.  Asynchronous on the stream: the positions
 * are complete when the stream is. */
int rod_step_io(rod_handle h, int n_steps, const float* drive, float* pos_out, void* stream);

/* Bind rod `inner` (guidewire) inside rod `outer` (catheter) of the same handle as a pair
 * stepped together in one thread block (Section 3.4).  mode 0: no interaction (v0);
 * 1: one-way binding, the outer rod is not moved (v1); 2: two-way binding (v2).  Binding
 * constraints are distance constraints of rest length zero (Section 2.1 "Constraints"),
 * applied after every constraint iteration in two colors: inner node i is bound to the
 * outer centreline point at arclength (i + beta) l0, where beta is slot 3 of the inner
 * rod's drive row (its insertion relative to the outer rod, in segments; read once per
 * rod_step).  Both rods must be inextensible with equal l0, dt and n_iters and at most
 * 1024 nodes; a rod can be in one pair.  Pairs are not supported by rod_rollout and
 * rod_adjoint.  Synchronous (rebuilds the launch plan). */
int rod_bind(rod_handle h, int outer, int inner, int mode);

/* Collision with an analytic vessel for rod `rod` (contact constraints C_c with Coulomb
 * friction, Section 2.1 "Constraints", iterated with the distance constraints as in
 * Section 3.3; an analytic tube stands in for the paper's vessel meshes).
 * tube: 8 host doubles (cx, cy, cz, Rc, Rt, mu, enable, 0): the vessel centreline is the
 * circle of radius Rc about (cx, cy) in the plane z = cz, its inner radius Rt > rod radius,
 * mu >= 0 the friction coefficient; enable = 0 removes the vessel.  Every constraint
 * iteration, after the distance sweeps, each dynamic node with predicted centreline offset
 * |(r - c) + dt v| > Rt - radius gets the normal velocity change that puts it on the wall
 * and a tangential velocity cut of at most mu times that change.
 * Errors: CORDE_ERR_ARG for a bad index, NULL tube, Rc <= 0, Rt <= rod radius or mu < 0;
 * CORDE_ERR_UNSUPPORTED for an extensible rod (n_iters = 0: no constraint iterations) or a
 * rod bound in a pair (rod_bind likewise refuses rods inside a vessel).  rod_adjoint
 * refuses handles with a vessel (contact is not differentiated).  Synchronous. */
int rod_set_tube(rod_handle h, int rod, const double* tube);

/* Self-collision of rod `rod` (contact constraints C_c for self-collisions with Coulomb
 * friction, Section 2.1 "Constraints"; bounding-sphere broad phase and sphere-sphere
 * narrow phase of "Collisions and self-collisions").
 * params: 2 host doubles (mu, enable): mu >= 0 the friction coefficient between strands;
 * enable = 0 turns it off.  Every mass point carries a sphere of the rod radius r.  Once
 * per step the pairs (i, j) with |i - j| >= max(2, floor(2 r / l0) + 1) and
 * |r_i - r_j| < 3 r are found; in every constraint iteration, after the distance sweeps
 * and the vessel contact, each pair whose predicted distance is below 2 r gets the
 * impulse that separates the predicted spheres, with a tangential cut of at most mu times
 * the normal change, and each mass point takes the penetration-weighted mean of its
 * pairs' velocity changes (one Jacobi pass).  The rod then runs in its own kernel (one
 * block, two elements per thread up to 512 nodes, four beyond).
 * Errors: CORDE_ERR_ARG for a bad index, NULL params or mu < 0; CORDE_ERR_UNSUPPORTED for
 * an extensible rod, a rod of more than 1024 nodes, a rod bound in a pair, or a handle
 * with a mailbox.  rod_rollout, rod_adjoint, rod_mailbox_enable and rod_bind refuse
 * self-colliding rods.  Synchronous. */
int rod_set_self_collision(rod_handle h, int rod, const double* params);

/* Self-collision statistics of rod `rod` from its last launch, into 5 host ints:
 * candidate pairs at the last detection, the most candidates j > i of one mass point i,
 * pairs whose spheres overlapped at the last detection, an overflow flag (bit 0 when
 * some mass point had more than 16 candidates above it, bit 1 when the rod had more than
 * 3 N candidate pairs, bit 2 when a mass point touched more than 16 others in one
 * iteration: the excess is dropped; bit 3 when a skin list overflowed, so that the next
 * step built it again instead of filtering it (the candidates stay exact); sticky until rod_set_self_collision), and the number of
 * skin-list builds in the launch.  Rods held by blocks of up to 512 nodes keep a skin
 * list (in device memory from one launch to the next): the detection runs with the reach
 * grown by 2 s (s = 1.5 r) and later steps test only the listed partners at the plain
 * reach, until a mass point has moved more than s since the list was built; the
 * candidate pairs are those of the full detection.  Synchronous. */
int rod_self_collision_stats(rod_handle h, int rod, int* out);

/* Copy the drive input [n_rods][8] (host or device) into the handle. */
int rod_set_input(rod_handle h, const float* drive, void* stream);

/* Copy the state out.  Each destination is [n_elements][4] float, element-indexed,
 * host or device, or NULL to skip:
 *  pos4   (x, y, z, inverse inertial node mass; 0 for a kinematic node)
 *  quat4  (x, y, z, w); the frame slot of each rod's last element is unused
 *  vel4   (vx, vy, vz, 0)
 *  omega4 (wx, wy, wz, 0), body frame; last element of each rod unused */
int rod_get_state(rod_handle h, float* pos4, float* quat4, float* vel4, float* omega4, void* stream);

/* Overwrite the state (same layouts; pos4.w is ignored, masses stay).  NULL skips. */
int rod_set_state(rod_handle h, const float* pos4, const float* quat4, const float* vel4,
                  const float* omega4, void* stream);

/* Sizes of the batch. */
int rod_info(rod_handle h, int* n_rods, int64_t* n_elements);

/* Derived constants (synchronous).  per_rod: [n_rods][16] host doubles
 *  l0, A, I, K1, K2, K3, Ks, Kp, mass_scale, inertia_scale, m_interior, J1, J2, J3,
 *  w_interior, 0.   per_joint: [n_elements][8] host floats (K1, K2, K3, 0, u-hat x, y,
 *  z, 0) for joint i between frames i and i+1; NULL skips either. */
int rod_get_derived(rod_handle h, double* per_rod, float* per_joint);

/* Override the per-joint stiffness and intrinsic Darboux vectors: [n_elements][8]
 * floats in the per_joint layout of rod_get_derived (host or device). */
int rod_set_material(rod_handle h, const float* per_joint, void* stream);

/* Per-rod diagnostics (synchronous): out [n_rods][4] host doubles =
 *  max |l_j / l0 - 1| over segments, max ||q_j| - 1|, number of non-finite state
 *  values, elastic energy (bend + penalty + stretch, FP64 accumulation).
 * Returns CORDE_ERR_NONFINITE if any rod holds a non-finite value. */
int rod_diagnostics(rod_handle h, double* out);

/* Kernel variants: elements per thread (ept) and threads per block (nt).  A rod of at
 * most 2048 nodes runs in one thread block; a longer one (up to 32768 nodes) is spread
 * over a cluster of `cluster` blocks that exchange border elements through distributed
 * shared memory and synchronise with cluster barriers (the GB300 form of the paper's
 * multi-block kernel, Section 2.2).  rod_set_plan forces one block variant for every rod
 * it can hold (ept = 0 restores the default plan); rod_set_plan_cluster forces a cluster
 * variant (ept, nt) in {(2,256), (4,256), (4,512)}, cluster 2..16, for every rod it can
 * hold; rod_autotune times the block variants that hold each length bin on the current
 * state (saved and restored) and keeps the fastest per bin.  rod_get_plan writes
 * [n_rods][3] ints (ept, nt, blocks; 0 = one block, C >= 2 a cluster of C blocks, -C a
 * cooperative grid of C blocks, see rod_set_plan_grid).  Synchronous. */
int rod_set_plan(rod_handle h, int ept, int nt);

/* Launch overlap (on by default): the stepping kernels are launched with programmatic
 * stream serialisation, so a launch is scheduled while the stream's previous stepping
 * kernel still runs and starts stepping as soon as that kernel's writes are visible (each
 * kernel waits for them before its first global access).  Results are bit for bit those
 * of ordinary launches; enable = 0 switches it off (e.g. to time the launch gap).
 * enable must be 0 or 1 (CORDE_ERR_ARG otherwise).  Host-side only. */
int rod_set_launch_overlap(rod_handle h, int enable);
int rod_set_plan_cluster(rod_handle h, int ept, int nt, int cluster);
/* A rod longer than a 16-block cluster holds (32768 nodes) runs on a cooperative grid
 * of `blocks` blocks (the paper's multi-block kernel, Section 2.2, over the whole GPU):
 * each block's first and last thread publish their exchange slots in global memory and
 * every exchange barrier is a grid sync; the runtime launches the grid only when all its
 * blocks are resident at once, so a sync never waits on a block that is not running.
 * rod_create gives such a rod 2048 nodes per block (ept 4, nt 512); the longest rod is
 * 2048 x the blocks the device holds at once (one per SM at nt 512).
 * rod_set_plan_grid forces the grid form of a cluster variant (ept, nt) in {(2,256),
 * (4,256), (4,512)} with `blocks` >= 2 blocks for every rod it can hold (the same
 * arithmetic as the cluster form: the same results bit for bit).  rod_get_plan reports
 * -blocks for a rod on a grid.  CORDE_ERR_UNSUPPORTED when the rods' blocks exceed what
 * the device holds at once, or with the mailbox (not available for rods on a grid).
 * Synchronous. */
int rod_set_plan_grid(rod_handle h, int ept, int nt, int blocks);
int rod_autotune(rod_handle h, int n_steps, void* stream);

/* Pick the number of time steps per launch, among n_candidates values (each >= 1), with
 * the shortest time per step for this handle's plan: a launch spreads its load, store and
 * launch latency over its steps, while the host's next input waits for the launch.  Each
 * candidate runs ceil(min_steps / candidate) launches from the same state (restored
 * afterwards, with the step count); two passes over the candidates, the second counts.
 * *best receives the winner.  Not with a mailbox.  Synchronous. */
int rod_autotune_steps(rod_handle h, const int* candidates, int n_candidates, int min_steps, int* best,
                       void* stream);
int rod_get_plan(rod_handle h, int* plan);

/* When one rod_step needs several kernel launches (rods of several length bins, bound
 * pairs), rod_step captures them once into a CUDA graph whose kernels run concurrently
 * and replays it (re-captured when n_steps or the plan changes; the drive is first copied
 * into an internal buffer the graph reads).  mode 0: never use a graph; 1: when more than
 * one launch is needed (default); 2: always.  The first rod_step after a change captures
 * on an internal stream: do not call it inside a caller's own stream capture. */
int rod_set_graph_mode(rod_handle h, int mode);

/* Mailbox of running launches (Section 2.2 and 3.1: the haptic thread writes the device's
 * state into the running kernel and reads the force feedback back, at a rate higher than
 * the kernel launches, through pinned memory while the kernel runs).  While enabled,
 * every rod_step launch polls the input every `period` steps (one non-blocking read of a
 * seqlock in mapped pinned host memory by the thread owning the rod's base; a torn or
 * unchanged input is skipped, nothing waits) and writes, every `period` steps, the base
 * and tip node's position and velocity to two feedback records per rod.  Each input a
 * rod picks up is logged as (global step, input sequence number), up to log_capacity
 * entries, so a run can be replayed exactly.
 *  rod_mailbox_enable   allocates the mapped buffers (synchronous); not with bound pairs.
 *  rod_mailbox_write    host-side seqlock write of [n_rods][8] drive rows (as rod_step's
 *                       drive); safe while kernels run; the k-th write gets sequence 2k.
 *  rod_mailbox_read     consistent copy of the records: out [n_rods][2][8] 32-bit words
 *                       (seq, step, x, y, z, vx, vy, vz as float bits); record 0 the base,
 *                       1 the tip; seq 0 means not written yet.  Safe while kernels run.
 *  rod_mailbox_log      copies min(count, capacity) (step, seq) pairs to out [capacity][2],
 *                       returns the count and clears the log (synchronous).
 *  rod_mailbox_disable  frees the mailbox (synchronous).
 *  rod_mailbox_positions_enable  (enable != 0) every rod additionally publishes all its
 *                       positions every `period` steps into mapped pinned host memory,
 *                       into a ring of 4 snapshot slots followed by a publication count
 *                       (the graphics/haptic thread pulls the whole rod while the kernel
 *                       runs; a slot is rewritten only after the count that retires it
 *                       is visible, so the host has 3 periods to copy one); allocates
 *                       4 x n_elements x 16 B of mapped memory (synchronous); needs
 *                       rod_mailbox_enable first.
 *  rod_mailbox_positions  consistent copy of rod `rod`'s latest snapshot: out [N][4]
 *                       floats (x, y, z, inverse mass), *step the global step it was
 *                       taken after (-1: none yet); out NULL: *step only, nothing copied
 *                       (a cheap poll).  Host-only and non-blocking for the device; a
 *                       copy during which the count advanced by 3 or more is retried,
 *                       CORDE_ERR_BUSY after 10000 tries.
 * With the mailbox enabled rod_step launches directly (no graph).  rod_steps_done: steps
 * taken by rod_step on this handle (the log's step index). */
int rod_mailbox_enable(rod_handle h, int period, int log_capacity);
int rod_mailbox_write(rod_handle h, const float* drive);
int rod_mailbox_read(rod_handle h, unsigned* out);
int rod_mailbox_log(rod_handle h, int* out, int capacity, int* count);
int rod_mailbox_disable(rod_handle h);
int rod_mailbox_positions_enable(rod_handle h, int enable);
/* Lock-step haptic loop (enable != 0): at every poll point (every `period` steps) the
 * thread owning a rod's base waits for a new input instead of skipping when there is
 * none, so each input drives exactly the next `period` steps; the rod's other threads
 * wait at a block barrier (a cluster barrier for a rod on a cluster).  The wait is
 * bounded by timeout_us of GPU time (checked with the GPU's global timer, backing off
 * between reads); when it runs out the launch stops stepping at that point, stores its
 * state and sets bit 0 of the mailbox status.  The host still counts the launch's n_steps
 * in rod_steps_done.  Synchronous. */
int rod_mailbox_lockstep(rod_handle h, int enable, int timeout_us);
/* Mailbox status word, cleared by the read: bit 0 = a lock-step wait ran out. */
int rod_mailbox_status(rod_handle h, unsigned* status);
int rod_mailbox_positions(rod_handle h, int rod, float* out, long long* step);
/* One tick of a haptic loop in one call: writes drive (as rod_mailbox_write; NULL: no
 * write), then spins on the host until rod `rod`'s newest position snapshot was taken
 * after a global step >= target_step, and copies it as rod_mailbox_positions does (out
 * [N][4] host floats, *step its step).  Only the snapshot header is polled while waiting.
 * Errors: CORDE_ERR_ARG (NULL out or step, snapshots not enabled, bad rod, timeout_us <
 * 0); CORDE_ERR_BUSY when timeout_us microseconds pass first or the mailbox status shows
 * that a lock-step wait of the kernel ran out (the status word is left set). */
int rod_mailbox_exchange(rod_handle h, const float* drive, int rod, long long target_step, float* out,
                         long long timeout_us, long long* step);
/* One tick of a closed haptic loop in lock-step (Section 2.2: input and feedback
 * exchanged with the running kernel every haptic frame): spins on the host until rod
 * `rod`'s newest position snapshot was taken after a global step >= target_step, then
 * writes next_drive (as rod_mailbox_write; NULL: no write) at once, so that the kernel's
 * lock-step wait for the next tick ends while the host still copies, then copies the
 * snapshot as rod_mailbox_positions does (out [N][4] host floats, NULL: none; *step its
 * step).  The drive of tick k + 1 thus follows the end of tick k, with no host code
 * between the two.  Errors as rod_mailbox_exchange (NULL step, snapshots not enabled,
 * bad rod, timeout_us < 0: CORDE_ERR_ARG; the timeout or a lost lock-step wait:
 * CORDE_ERR_BUSY, and next_drive is not written). */
int rod_mailbox_tick(rod_handle h, int rod, long long target_step, const float* next_drive, float* out,
                     long long timeout_us, long long* step);
int64_t rod_steps_done(rod_handle h);

/* Number of kernel launches the last rod_step enqueued (kernel nodes of the graph when
 * the graph path ran). */
int rod_last_launch_count(rod_handle h);

/* Forward rollout recorded for the adjoint: n_steps time steps with the drive last given
 * to rod_set_input held constant, storing the state every ckpt_every steps (checkpoints
 * kept by the handle) and, if pos_traj is not NULL, the node positions after every step
 * into pos_traj [n_steps][n_elements][4] (device memory; .w = inverse mass).  When every
 * rod has at most 512 nodes the launches use the adjoint's kernel layout.  The handle's
 * state advances to step n_steps.  (Not in the paper: this and rod_adjoint provide the
 * gradients of a loss on the trajectory.) */
int rod_rollout(rod_handle h, int n_steps, int ckpt_every, float* pos_traj, void* stream);

/* Reverse-mode gradient of a loss L(trajectory) through the last rod_rollout (hand-written
 * adjoint of the step of Fig. 5, checkpoint-and-recompute).  Input dL_dpos_traj
 * [n_steps][n_elements][4] device array: dL/d(position after step t) in .xyz (or NULL for
 * zero).  Outputs, [n_elements][4] device arrays, any may be NULL:
 *  dL_dK      per-joint stiffness (K1, K2, K3, 0) of joint i (frames i, i+1)
 *  dL_duhat   per-joint intrinsic Darboux vector (x, y, z, 0)
 *  dL_dvel0, dL_dpos0   initial node velocities / positions (xyz, 0)
 *  dL_dquat0  initial frames (x, y, z, w components), dL_domega0 initial body angular velocities
 * Rods of at most 512 nodes; shared memory bounds the constraint iterations (68 for
 * rods of up to 256 nodes, 30 for longer ones).  The material, drive and state set between rod_rollout and
 * rod_adjoint must not change.  CORDE_ERR_UNSUPPORTED when the limits are exceeded. */
int rod_adjoint(rod_handle h, const float* dL_dpos_traj, float* dL_dK, float* dL_duhat, float* dL_dvel0,
                float* dL_dpos0, float* dL_dquat0, float* dL_domega0, void* stream);

/* How the last rod_adjoint ran its largest launch, into 7 host ints: the mode (0
 * recompute; 1 record mode with one sweep buffer in shared memory; 2 record mode with
 * two, the copy of a step's records overlapping the reverse of the step after it),
 * threads per block, resident blocks per SM (occupancy API, with the launch's registers
 * and shared memory; 1 when pipelined), blocks of the launch (one per rod, two when
 * pipelined), the device's SMs, 1 when the records use the compact layout (see
 * rod_set_adjoint_record_budget), and 1 when the reverse pass was pipelined (see
 * rod_set_adjoint_pipeline); blocks / (blocks per SM x SMs), rounded up, is the number
 * of waves.  Host-side only (zeros before the first rod_adjoint). */
int rod_adjoint_info(rod_handle h, int* out);

/* Scratch budget of rod_adjoint's record mode (default 1 GiB).  Within a checkpoint
 * segment the reverse pass needs every step's velocities before each constraint
 * half-sweep.
 *  - Record mode (the scratch fits in `bytes`): one forward pass over the segment keeps
 *    them in device memory, 2 n_iters x 12 B per node and step (beside the segment's
 *    states, 48 B per node and step).  A launch with more rods than the GPU has SMs (or one whose
 *    full records do not fit) keeps the compact layout instead: the velocities before
 *    the first even and every odd half-sweep, (n_iters + 1) x 12 B per node and step;
 *    its reverse pass repeats each odd half-sweep on its record to get the input of the
 *    next even one.  The reverse pass streams the records back with asynchronous
 *    copies, into two shared-memory buffers (the copy of a step's records overlaps the
 *    reverse of the step after it) or into one when two do not fit or when one buffer
 *    lets more blocks share an SM and so runs the launch in fewer waves.
 *  - Recompute mode (otherwise, and always with bytes = 0): every step is run forward
 *    again before its reverse.
 * All modes give the same gradients bit for bit.  bytes >= 0 (CORDE_ERR_ARG otherwise).
 * Host-side only. */
int rod_set_adjoint_record_budget(rod_handle h, long long bytes);

/* Pipelined reverse pass (enable != 0, the default).  A record-mode launch with the full
 * layout and two sweep buffers whose rods each find two free SMs (2 x rods <= SMs) runs
 * every rod on a cluster of two blocks: the first block records the checkpoint segments
 * (last first), the second reverses each one a segment later, so that recording and
 * reversing overlap; one cluster barrier per segment hands a segment's scratch over.  It
 * takes twice the record scratch (segment states and records in two sets, by segment
 * parity), within the record budget.  The gradients are the same bit for bit.  Host-side
 * only. */
int rod_set_adjoint_pipeline(rod_handle h, int enable);

/* Gradient of one rod's rollout without any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc where
 * they need a gradient - a haptic or control loop under a real-time budget (an allocation
 * can stall and synchronise the device), or an application whose device memory is
 * owned by its own pool.  It runs the recorded rollout (as rod_rollout) and the reverse
 * pass (as rod_adjoint) of a single rod described like rod_create's arguments, keeping
 * every intermediate in one static 16 MiB array that is part of the library image (every
 * GPU that loads the library holds it until the process exits).
 *  params         one rod (host).  Inputs, device memory in rod_create's layouts: pos [N][3],
 *                 quat [N-1][4], rest_quat, vel, omega, stiff_mul (NULL allowed as in
 *                 rod_create), drive [8] or NULL (zero).
 *  dL_dpos_traj   [n_steps][N][4] device, dL/d(position after step t), or NULL.
 *  Outputs (device, [N][4] floats, NULL skips): pos_traj [n_steps][N][4] positions after
 *                 every step; dL_dK, dL_duhat, dL_dvel0, dL_dpos0 as in rod_adjoint.
 * Limits: N <= 512 and (ceil(n_steps / ckpt_every) + min(ckpt_every, n_steps)) * 64 * N
 * bytes plus about 100 * N bytes must fit in 16 MiB; larger requests return CORDE_ERR_ARG
 * with the size needed.  It calls no cudaMalloc, cudaFree or other allocating routine.
 * The first call on each device, with that device current, looks up the array's device
 * address (cudaGetSymbolAddress) and loads every kernel the entry point can launch (with
 * lazy module loading, the CUDA default, a kernel's first launch would load its module,
 * which takes device memory): make that first call before any stream capture and outside
 * the real-time part of the program; later calls load nothing.  Every call
 * shares the one array and overwrites it; calls that overlap on the GPU (other streams,
 * other host threads) race and give wrong results.  Asynchronous on `stream`. */
int rod_adjoint_noalloc(const RodParams* params, const float* pos, const float* quat, const float* rest_quat,
                        const float* vel, const float* omega, const float* stiff_mul, const float* drive,
                        int n_steps, int ckpt_every, const float* dL_dpos_traj, float* pos_traj, float* dL_dK,
                        float* dL_duhat, float* dL_dvel0, float* dL_dpos0, void* stream);

/* Empty-barrier floor (synchronous): ns per barrier over n_iters back-to-back barriers
 * of one scope in a single launch.  The paper's multi-block kernel pays an inter-block
 * barrier per data exchange (Section 2.2, Fig. 5); these floors are the reference for a
 * step kernel's latency per step.
 *  scope 0: __syncthreads in one block of `threads` threads
 *  scope 1: __syncwarp in one warp
 *  scope 2: cluster barrier across `cluster` (<= 16) blocks of `threads` threads
 *  scope 3: cooperative grid sync across `cluster` blocks per SM on every SM (the
 *           runtime rejects the launch if they cannot be co-resident; it never hangs)
 * Returns CORDE_ERR_ARG for bad sizes, CORDE_ERR_CUDA if the launch is rejected. */
int rod_barrier_floor(int scope, int threads, int cluster, int n_iters, double* ns_per_barrier, void* stream);

/* Device facts read from the runtime (current device): number of SMs and resident
 * threads per SM; either pointer may be NULL.  CORDE_ERR_UNSUPPORTED without a GPU. */
int rod_device_info(int* n_sms, int* max_threads_per_sm);

/* FP32 arithmetic peak of the current device, measured (synchronous): the roofline that
 * the step kernels' per-element arithmetic (the force and torque evaluation of Eq. 2, 3,
 * 8 and the constraint impulses of Section 2.1) is compared against.  blocks_per_sm x
 * (number of SMs) blocks of `threads` threads (a multiple of 32, <= 1024) each run 8
 * independent fused multiply-add chains of n_iters steps; packed = 1 uses float2 chains
 * through the paired-lane FMA (two FMAs per lane and instruction).  One untimed launch,
 * then one timed with CUDA events on `stream`; *tflops receives 2 (packed: 4) x 8 x
 * n_iters x threads x blocks flops over that time.  CORDE_ERR_ARG for bad sizes. */
int rod_fp32_peak(int packed, int blocks_per_sm, int threads, int n_iters, double* tflops, void* stream);

/* Free the device state (synchronises the device first).  NULL is ignored. */
void rod_destroy(rod_handle h);

/* Static description of an error code; message of the last failing call (thread-local). */
const char* rod_strerror(int code);
const char* rod_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CORDE_H_ */

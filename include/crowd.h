/*
 * crowd.h -- C ABI of the batched ORCA crowd step on GB300 (sm_103a).
 *
 * The library moves the dynamic agents of many independent scene instances
 * ("environments") one simulation step at a time: pedestrians avoid each
 * other and the static segment obstacles of their block with ORCA, and each
 * environment may hold one robot agent whose velocity is commanded from
 * outside.  This is the per-step update of the paper's "Interactive Dynamics
 * Generation" (Sec. 3.2): sample start and end points per agent, then adjust
 * every agent in real time from proximity and relative velocity, across many
 * parallel environments, reacting to the trained robot, all on the GPU.  The
 * collision-avoidance rule is the ORCA method the paper cites (van den Berg
 * et al., "Reciprocal n-body collision avoidance", ISRR 2011).
 *
 * One step, per agent, in order:
 *   (A0) preferred velocity toward the goal; the robot takes its command;
 *   (A1-A2) neighbours: agents of the same environment within the neighbour
 *        distance R, ordered by (FP64 squared distance, index), first K;
 *   (A3) one reciprocal half-plane per neighbour (truncated velocity obstacle,
 *        horizon tau; horizon dt when already overlapping);
 *   (A4) one half-plane per static segment within r + tau_obst * v_max;
 *   (A5) the velocity closest to the preferred one inside the speed disk and
 *        all half-planes; when none exists, the velocity of least maximal
 *        penetration of the agent half-planes (segment half-planes stay hard),
 *        ties broken by closeness to the preferred velocity;
 *   (A6) explicit Euler: v <- v*, p <- p + dt v*; every agent moves from the
 *        step-start state of its environment.
 *
 * Conventions
 *   - SI units.  Agents are stored environment-major: environment e owns the
 *     agents [sum_{f<e} agents_per_env[f], ... + agents_per_env[e]).
 *     Segments likewise, with segs_per_env.
 *   - Every buffer passed in is copied during the call; the caller keeps
 *     ownership.  ptr_kind says whether a pointer is host (CROWD_HOST) or
 *     device (CROWD_DEVICE) memory; device pointers must be on the handle's
 *     device.
 *   - All calls enqueue on the handle's CUDA stream and return before the GPU
 *     finishes, except crowd_read_*, crowd_synchronize and crowd_destroy,
 *     which wait for the stream.
 *   - No exception crosses this interface: every call returns a crowd_status;
 *     crowd_last_error() gives a message for the calling thread's last failure.
 *   - A handle is not thread-safe: serialise calls on the same handle.
 *   - Device-side faults of the algorithm (more than the supported number of
 *     segment half-planes for one agent) set an error word that the next
 *     synchronising call reports as CROWD_EDEVICE.
 */
#ifndef CROWD_H
#define CROWD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct crowd_ctx* crowd_t;

typedef enum {
    CROWD_OK = 0,
    CROWD_EINVAL = 1,  /* bad argument (NaN/Inf input, r <= 0, v_max < 0, K > 32, R <= 0, dt <= 0, ...) */
    CROWD_ENOMEM = 2,  /* device allocation failed */
    CROWD_ECUDA = 3,   /* a CUDA runtime call failed */
    CROWD_EDEVICE = 4, /* the device error word was set by a kernel */
    CROWD_ESTATE = 5   /* call out of order (e.g. a handle that failed earlier) */
} crowd_status;

enum { CROWD_HOST = 0, CROWD_DEVICE = 1 };

/* crowd_params.flags */
enum {
    CROWD_FLAG_EXPORT_NEIGHBORS = 1, /* keep the neighbour lists of the last step (crowd_read_neighbors) */
    CROWD_FLAG_STATS = 2,            /* accumulate rollout statistics (crowd_read_stats) */
    CROWD_FLAG_COUNT_WORK = 4,       /* count the algorithm's work items (crowd_read_work) */
    CROWD_FLAG_FORCE_TILED = 8,      /* run every environment on the tiled (global-memory) path; by
                                        default only environments of more than 2048 agents do */
    CROWD_FLAG_VELOCITY_SEGMENTS = 16 /* segment half-planes tangent to the segment's truncated velocity
                                         obstacle at its boundary point nearest the agent's current
                                         velocity (full responsibility; the obstacle treatment of the
                                         method the paper cites, each segment on its own) instead of at
                                         its point nearest 0 */
};

/* Work counters (CROWD_FLAG_COUNT_WORK), summed over all agents and steps
 * since the handle was created: the units the algorithmic operation count of
 * one step is built from. */
typedef struct {
    uint64_t agent_steps;    /* agent updates performed */
    uint64_t candidates;     /* neighbour candidates tested (agents of the 3x3 cell block) */
    uint64_t agent_lines;    /* reciprocal agent half-planes built */
    uint64_t obstacle_lines; /* static-segment half-planes built */
    uint64_t segment_tests;  /* segment distance evaluations */
    uint64_t lp_checks;      /* half-plane checks of the incremental LP */
    uint64_t lp_solves;      /* 1D sub-solves (a line violated by the current point) */
    uint64_t lp_solve_lines; /* previous lines scanned by those sub-solves */
    uint64_t fallbacks;      /* agents whose LP was infeasible */
    uint64_t pairs_in_range; /* candidates j != i within R (FP64 key < R^2): what an exact search must test */
} crowd_work;

/* Maximum number of neighbours K. */
#define CROWD_MAX_NEIGHBORS 32
/* Maximum number of segment half-planes for one agent in one step. */
#define CROWD_MAX_OBSTACLE_LINES 64

typedef struct {
    float time_horizon;         /* tau > 0, seconds (agents) */
    float time_horizon_obst;    /* tau_obst >= 0, seconds (static segments); 0 means tau */
    float neighbor_dist;        /* R > 0, metres */
    int32_t max_neighbors;      /* K in [0, 32] */
    float robot_responsibility; /* share of the avoidance an agent takes against the robot, in [0, 1]; ORCA's 1/2 */
    int32_t flags;              /* CROWD_FLAG_* */
} crowd_params;

/* Per-environment rollout statistics (only with CROWD_FLAG_STATS), summed over
 * the post-integration state of every step since the last reset:
 *   agent_collisions: pairs i < j with |p_i - p_j| < r_i + r_j - 0.001,
 *   segment_collisions: (agent, segment) pairs closer than r_i - 0.001
 *     (a collision is a penetration deeper than 1 mm),
 *   speed_sum: sum of |v| over the non-robot agents,
 *   steps: number of steps accumulated.
 * These are the collision indicator and speed of the paper's metric table
 * (Appendix, "Evaluation Metrics"). */
typedef struct {
    int64_t agent_collisions;
    int64_t segment_collisions;
    double speed_sum;
    int64_t steps;
} crowd_env_stats;

/* Create a batch of n_envs environments on the current CUDA device.
 * Paper: Sec. 3.2 -- the dynamic agents of many parallel environments, each
 * with its radius and maximum speed, the ORCA time horizon and neighbour
 * distance, the static objects of the generated scene (segments) and the
 * trained robot as one more agent; Sec. 3.3 -- environments of different
 * sizes side by side in one batch.
 *   agents_per_env [n_envs]     agents of each environment (>= 0)
 *   radii, max_speeds [N]       r > 0, v_max >= 0 (N = total agents)
 *   pref_speeds [N] or NULL     preferred walking speed; NULL means v_max
 *   init_pos [N][2]             start positions; velocities start at 0
 *   robot_index [n_envs] or NULL environment-local index of the robot agent, -1 for none
 *   segs_per_env [n_envs] or NULL, segments [S][4] (ax, ay, bx, by) static segment obstacles; zero-length rejected
 *   p                           parameters (copied)
 *   cuda_stream                 cudaStream_t to enqueue on (NULL: the legacy default stream)
 *   out                         receives the handle; owns all its device memory
 * All pointers here are host pointers.  Goals start at the initial positions. */
crowd_status crowd_create(int32_t n_envs, const int32_t* agents_per_env, const float* radii,
                          const float* max_speeds, const float* pref_speeds, const float* init_pos,
                          const int32_t* robot_index, const int32_t* segs_per_env, const float* segments,
                          const crowd_params* p, void* cuda_stream, crowd_t* out);

/* Goals [N][2] (fixed goals; removes a goal queue).
 * Paper: Sec. 3.2 -- every agent gets a sampled end point and walks toward
 * it (the preferred velocity of step A0). */
crowd_status crowd_set_goals(crowd_t h, const float* goals, int32_t ptr_kind);

/* Goal queues (continuing walks after arrival; the paper's agents walk
 * between sampled start and end points, Sec. 3.2, and the simulation runs on
 * past their arrival).  Agent i walks to goals[i][0], then goals[i][1], ...:
 * at the start of every step, an agent (not the robot) whose position p lies
 * within its radius r of its current goal g, |g - p|^2 <= r^2 (decided as an
 * FP64 evaluation of the FP32 values decides it), moves on to its next goal,
 * which it steers to from that step on.  After the last goal the queue starts
 * again when `cyclic` != 0; otherwise the agent keeps its last goal.
 *   n_goals: goals per agent, 1..CROWD_MAX_GOALS; goals [N][n_goals][2],
 *            host or device (copied).
 * The first goal of each queue becomes the agent's current goal and every
 * counter is reset to 0; crowd_set_goals removes the queue.  Waits for the
 * handle's stream; allocates device memory on the first call. */
#define CROWD_MAX_GOALS 64
crowd_status crowd_set_goal_queue(crowd_t h, int32_t n_goals, const float* goals, int32_t cyclic, int32_t ptr_kind);

/* Goal pools (the paper samples agents' start and end points on the
 * traversable ground, Sec. 3.2; crowd_map_sample draws such points): at the
 * start of every step an agent (not the robot, not a car) within its radius
 * of its goal, decided as for goal queues, draws its next goal inside the
 * kernel from its environment's pool: with k the draws it made so far,
 * u = Philox4x32-10(counter (g, k, 0, 0), key (seed low 32 bits, seed high
 * 32 bits)), g its global index, the point floor(u.x n / 2^32) of the n
 * points of its environment (none drawn when n = 0).
 *   pool_start [n_envs + 1] host (pool_start[0] = 0, non-decreasing): the
 *   points of environment e are points[pool_start[e] .. pool_start[e + 1]),
 *   points [P][2] host.  NULL pool_start removes the pool.
 * Replaces a goal queue (and crowd_set_goals or crowd_set_goal_queue
 * replace the pool); the counters restart at 0, current goals stay; removes
 * the episodes.  CROWD_EINVAL for a bad layout or NaN/Inf.  Copies; waits. */
crowd_status crowd_set_goal_pool(crowd_t h, const int32_t* pool_start, const float* points, uint64_t seed);

/* Host copy [N] of how many goals each agent has moved past (queue) or drawn
 * (pool) since they were set (0 without either).  Waits.
 * Paper: Sec. 3.2 (end points sampled per agent); the counter is this
 * library's read-back of the goal queues and pools above. */
crowd_status crowd_read_goal_index(crowd_t h, int32_t* out);

/* Lane-following vehicles (the paper's city scenes run cars beside the
 * crowd under the Intelligent Driver Model of Treiber, Hennecke and Helbing,
 * 2000; Appendix "Data", and Sec. 3.2's vehicles among the dynamic agents).  Lanes are closed polylines: lane l has points
 * points[lane_start[l]..lane_start[l+1]) ([P][2], at least 2, no zero-length
 * segment; the last point joins the first).  Vehicle k (agents ascending) is
 * crowd agent `agent[k]` (global index, not a robot slot, at most
 * CROWD_MAX_VEHICLES_PER_ENV per environment, on either kernel), on lane `lane[k]` at arc position s[k] in [0, lane
 * length) with speed v[k] >= 0, IDM parameters params[k][6] = (desired
 * speed v0, time gap T, acceleration a, comfortable deceleration b, jam
 * distance s0, length), all > 0.  Each step, from the step-start state, a
 * car's leader is the nearest thing ahead on its lane: another car of the
 * lane (gap ds - (len_i + len_j)/2, approach rate v_i - v_j) or a crowd agent
 * within half_width + r of the lane and at most `lookahead` ahead (gap
 * ds - len_i/2 - r, standing still); acceleration
 * a (1 - (v/v0)^4 - (s_star / gap)^2), s_star = s0 + max(0, v T + v dv / (2 sqrt(a b))),
 * the interaction term dropped with nothing ahead, the gap floored at
 * 0.01 m; v' = max(0, v + acc dt), s' = s + v' dt (wrapped).  During the
 * step the car is its agent at p(s) moving at (p(s') - p(s)) / dt; every
 * other agent avoids it with full responsibility; it is left out of the
 * speed and goal statistics and of goal queues.  n_vehicles = 0 removes the
 * cars.  Copies everything; waits for the stream. */
#define CROWD_MAX_VEHICLES_PER_ENV 32
crowd_status crowd_set_vehicles(crowd_t h, int32_t n_lanes, const int32_t* lane_start, const float* points,
                                int32_t n_vehicles, const int32_t* agent, const int32_t* lane, const float* s,
                                const float* v, const float* params, float half_width, float lookahead);

/* Arc positions s [V] and speeds v [V] of the vehicles: written from the host
 * when `write` != 0 (s in [0, lane length), v >= 0), else read.  Waits.
 * Paper: Appendix "Data" (cars under the IDM beside the crowd); reading and
 * writing their state is this library's checkpoint of them. */
crowd_status crowd_vehicle_state(crowd_t h, int32_t write, float* s, float* v);

/* Episodes: environments start over inside multi-step calls, each on its own
 * schedule (the paper trains on many environments at once whose episodes
 * differ, Sec. 3.3).  The episode clock reads t = 0 at the next step after
 * this call.  Environment e with steps[e] > 0 starts over at the start of
 * every step t > 0 that is a multiple of steps[e], before anything else of
 * that step: its agent rows become those of init_state ([N][4], host or
 * device per ptr_kind; NULL: the state at this call), and its goals,
 * goal-queue counters and car arc states become those at this call.  The
 * state read after the step that ends an episode is the episode's last
 * state.  Statistics run on across starts: collisions count every
 * post-integration state (episode ends included, restored states not),
 * first-reach steps keep their first value.
 *   steps [n_envs] host, >= 0 (0: never; all 0 keeps the snapshot for
 *   crowd_restart_envs alone); NULL removes the episodes, as do
 *   crowd_set_goals, crowd_set_goal_queue and crowd_set_vehicles.
 * crowd_reset_stats leaves the episode clock running.  The serving loop and
 * crowd_step_noalloc have no episodes.  CROWD_EINVAL: steps[e] < 0, NaN/Inf
 * in a host init_state.  Copies; waits for the stream. */
crowd_status crowd_set_episodes(crowd_t h, const int32_t* steps, const float* init_state, int32_t ptr_kind);

/* Paper: Sec. 3.3 (episodes that differ per environment).
 * Per-environment reset mask: the environments with mask[e] != 0 start over
 * now, between calls, from the snapshot of crowd_set_episodes (agent rows,
 * goals, goal-queue counters, car arcs), as a scheduled start does; the
 * others keep their state.  For episodes that end on events (a collision, an
 * arrival) rather than after a fixed number of steps.  mask [n_envs] host
 * (copied).  CROWD_ESTATE without a snapshot; waits for the stream. */
crowd_status crowd_restart_envs(crowd_t h, const uint8_t* mask);

/* Full state [N][4] (px, py, vx, vy): resume from a checkpoint, or teacher
 * forcing from another simulator's state.
 * Paper: Sec. 3.2 -- the agents' positions and velocities, the state the
 * per-step adjustment reads. */
crowd_status crowd_set_state(crowd_t h, const float* state, int32_t ptr_kind);

/* Advance every environment by n_steps >= 1 steps of length dt > 0.
 * Paper: Sec. 3.2 -- every step each agent's velocity is adjusted in real
 * time from the proximity and relative velocity of the others (ORCA, steps
 * A0-A6 above), reacting to the trained robot, whose velocity is the action
 * given here; Sec. 3.3 -- all environments are stepped together on the GPU.
 * robot_vel [n_steps][n_envs][2] m/s, the robot command of each step
 * (entries of environments without a robot are ignored); NULL keeps every
 * robot at its current velocity. */
crowd_status crowd_step(crowd_t h, float dt, const float* robot_vel, int32_t ptr_kind, int32_t n_steps);

/* Copy the state [N][4] (px, py, vx, vy) out; waits for the stream.
 * Paper: Sec. 3.2 -- the adjusted agent positions (and velocities) that the
 * simulator hands to the rest of the platform each step. */
crowd_status crowd_read_state(crowd_t h, float* out, int32_t ptr_kind);

/* Neighbour lists [N][K] of the last step (environment-local indices, -1
 * padded), only with CROWD_FLAG_EXPORT_NEIGHBORS; waits for the stream.
 * Paper: Sec. 3.2 ("proximity": the agents each one reacts to, step A2). */
crowd_status crowd_read_neighbors(crowd_t h, int32_t* out, int32_t ptr_kind);

/* Host copies of the per-environment statistics [n_envs] and of the goal
 * reach step of every agent [N] (1-based global step index after which
 * |g - p| <= r first held, -1 if not yet); either may be NULL.  Waits.
 * Paper: Appendix "Evaluation Metrics" (collision indicator, speed, goal
 * reached). */
crowd_status crowd_read_stats(crowd_t h, crowd_env_stats* env_stats, int32_t* reach_step);

/* Host copy of the work counters (only with CROWD_FLAG_COUNT_WORK).
 * No counterpart in the paper: the units of the step's algorithmic
 * operation count (Sec. 3.2's step, counted for the roofline). */
crowd_status crowd_read_work(crowd_t h, crowd_work* out);

/* Kernels this handle's crowd_step calls have enqueued since it was created
 * (a replayed CUDA graph counts its kernels), into *out; host-side count, no
 * wait.  No counterpart in the paper: it lets a caller count the library's
 * launches inside a timed region. */
crowd_status crowd_read_launches(crowd_t h, int64_t* out);

/* Launch shape of the shared-memory-resident kernel (environments of up to
 * 2048 agents).  None of these changes results except coop_fallback, which
 * changes only the rounding of infeasible-LP fallbacks (both within the
 * 1e-4 m/s contract).
 *   block_threads: threads per CTA, a multiple of 32 in [32, 512], or 0 for
 *                  one thread per agent of the largest environment;
 *   coop_fallback: 0 = infeasible LPs are solved in place by their thread
 *                  (the default); 1 = queued and solved by whole warps after
 *                  the pass; 2 = queued and solved after the pass by one
 *                  thread each, spread over the warps so that no warp runs
 *                  two of them in turn (in place when the queue is full);
 *   cell_split:    s = 1, 2 or 3: grid cells >= R/s and a (2s+1)^2 cell
 *                  search (finer cells, fewer candidates per agent);
 *   lanes_per_agent: 1, 2, 4 or 8 lanes of a warp share each agent's work
 *                  (neighbour candidates, half-planes, LP intervals); with
 *                  more than one, fallbacks run in place; 0 means 1;
 *   agent_order:   one lane per agent: 0 = each warp takes a run of agents
 *                  in cell order, 1 = the lanes of a warp take agents
 *                  (warps) apart in cell order, which spreads a crowded
 *                  region over all warps.
 * block_threads 0 means one group of lanes per agent of the largest
 * environment, at most 512 threads.
 * The tiled path (environments of more than 2048 agents):
 *   tiled_queue:   1 = one persistent launch per step whose warps take work
 *                  items (32 agents in cell order of one environment) from a
 *                  counter shared by all tiled environments (the default);
 *                  0 = one CTA per tile of cells, its halo staged in shared
 *                  memory.  Both give the same bits. */
typedef struct {
    int32_t block_threads;
    int32_t coop_fallback;
    int32_t cell_split;
    int32_t lanes_per_agent;
    int32_t agent_order;
    int32_t tiled_queue;
} crowd_tuning;

/* Read / set the launch shape.  No counterpart in the paper (this
 * library's launch parameters for Sec. 3.2's step). */
crowd_status crowd_get_tuning(crowd_t h, crowd_tuning* out);
crowd_status crowd_set_tuning(crowd_t h, const crowd_tuning* t);

/* No counterpart in the paper (chooses this library's launch shape).
 * Time every tuning candidate (one lane per agent: block_threads
 * default/64/128/256/512 x coop_fallback 0 and 2 x cell_split 1-3 x
 * agent_order; 2, 4 and 8 lanes per agent: the default block and 512 threads
 * x cell_split 1-2; with tiled environments, tiled_queue 0 and 1) over
 * n_steps steps of length dt from the current state, keep
 * the fastest, and restore the state, statistics and counters.  Waits for the
 * stream; allocates temporary device memory.  `chosen` may be NULL. */
crowd_status crowd_autotune(crowd_t h, float dt, int32_t n_steps, crowd_tuning* chosen);

/* Zero the statistics and reach steps and restart the step counter at 0.
 * Paper: Appendix "Evaluation Metrics" (the statistics reset here). */
crowd_status crowd_reset_stats(crowd_t h);

/* Wait for all work enqueued on the handle; reports a device error word.
 * No counterpart in the paper (stream ordering of this library). */
crowd_status crowd_synchronize(crowd_t h);

/* Release the handle and its device memory (waits for the stream first).
 * No counterpart in the paper (resource lifetime of this library). */
crowd_status crowd_destroy(crowd_t h);

/* Number of agents / environments of a handle (0 for NULL).
 * Paper: Sec. 3.2-3.3 (agents per environment, parallel environments). */
int64_t crowd_num_agents(crowd_t h);
int32_t crowd_num_envs(crowd_t h);

/* ------------------------------------------------------------------------
 * Serving loop with continuous batching.  Rollout requests (one environment
 * each, with its own step count) are submitted at any time; crowd_server_tick
 * admits waiting requests first come first served into free slots while the
 * device-memory budget allows, advances every live request by up to
 * chunk_steps steps in one batched launch, and copies finished results back.
 * A request's result depends only on its own inputs, not on the batch it ran
 * in.  Not thread-safe.
 * ------------------------------------------------------------------------ */
typedef struct crowd_server_ctx* crowd_server_t;

typedef struct {
    int32_t max_slots;     /* requests resident at once, [1, 65536] */
    int32_t max_agents;    /* per request, [1, 2048] */
    int32_t max_segments;  /* per request, >= 0 */
    int32_t max_steps;     /* per request, >= 1 */
    size_t mem_budget;     /* bytes of request state admitted at once */
    int32_t chunk_steps;   /* steps per tick, >= 1 */
} crowd_server_config;

typedef struct {
    int32_t n_agents;
    const float* radii;        /* [n] > 0 */
    const float* max_speeds;   /* [n] >= 0 */
    const float* pref_speeds;  /* [n] or NULL (= max_speeds) */
    const float* init_pos;     /* [n][2]; velocities start at 0 */
    const float* goals;        /* [n][2] */
    int32_t robot_index;       /* -1 for none */
    int32_t n_segments;
    const float* segments;     /* [n_segments][4] */
    int32_t n_steps;
    const float* robot_vel;    /* [n_steps][2] or NULL (robot at rest) */
} crowd_request;

enum { CROWD_REQ_QUEUED = 0, CROWD_REQ_RUNNING = 1, CROWD_REQ_DONE = 2 };

typedef struct {
    int32_t waiting;
    int32_t live;
    size_t bytes_in_use;
} crowd_server_stats;

/* Serving: Sec. 3.3's many non-uniform environments, here as rollout
 * requests of different sizes admitted while others run.
 * Create a server on the current device (allocates its slot arena; all
 * pointers host).  dt is the step length of every request. */
crowd_status crowd_server_create(const crowd_params* p, float dt, const crowd_server_config* cfg, void* cuda_stream,
                                 crowd_server_t* out);
/* Validate and copy a request (host pointers); its id is written to *id.
 * Paper: Sec. 3.3 (one more non-uniform environment joins the batch). */
crowd_status crowd_server_submit(crowd_server_t s, const crowd_request* r, int64_t* id);
/* Retire the previous tick (waits for it), admit, and enqueue the next chunk.
 * Paper: Sec. 3.2-3.3 (all live environments stepped together on the GPU).
 * n_live: requests stepped by this tick; n_finished: requests the previous
 * tick completed.  Either may be NULL. */
crowd_status crowd_server_tick(crowd_server_t s, int32_t* n_live, int32_t* n_finished);
/* Paper: Sec. 3.2 (the adjusted agent states of a finished request).
 * Status of a request (CROWD_REQ_*); when done, its final state [n][4] is
 * copied to out_state (if not NULL) and the request is forgotten. */
crowd_status crowd_server_poll(crowd_server_t s, int64_t id, float* out_state, int32_t* status);
/* No counterpart in the paper (completion queue of the serving loop).
 * Ids of up to `cap` requests completed since the last call (oldest first);
 * *n receives how many were written.  Their results stay available to
 * crowd_server_poll. */
crowd_status crowd_server_finished(crowd_server_t s, int64_t* ids, int32_t cap, int32_t* n);
/* Waiting / live requests and bytes in use; release the server.
 * No counterpart in the paper (admission state and lifetime of this library). */
crowd_status crowd_server_info(crowd_server_t s, crowd_server_stats* out);
crowd_status crowd_server_destroy(crowd_server_t s);

/* ------------------------------------------------------------------------
 * Allocation-free step.  The paper has no counterpart: this entry point is
 * for callers that cannot call cudaMalloc -- code running inside another
 * framework's memory pool or under a fixed device-memory budget, real-time
 * loops that must not allocate after start-up, plug-ins handed only raw
 * device pointers.  It advances ONE environment by one step with the tiled
 * kernels and keeps every intermediate buffer (cell keys, ranks, counts and
 * starts, the state in cell order, per-cell segment lists) in one fixed
 * file-scope device array of about 7 MB that every GPU loading the library
 * holds until the process exits.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   - Limits: n_agents <= CROWD_NOALLOC_MAX_AGENTS; the grid over `box`
 *     (cells of at least neighbor_dist, at most 256 a side) <=
 *     CROWD_NOALLOC_MAX_CELLS cells; segment-cell list entries <=
 *     CROWD_NOALLOC_MAX_SEGMENT_CELLS.  Larger inputs fail with CROWD_EINVAL.
 *   - All calls share the array and it keeps the last call's contents: each
 *     call clears what must start at zero, but calls whose GPU work overlaps
 *     (other streams, other host threads) race on it -- serialise them.
 *   - The first call on a device looks up the array's address with that
 *     device current and sets a kernel attribute; make it before any stream
 *     capture.  Each call waits for the stream twice: to check the size of
 *     the segment lists, and at the end to read the device error word (an
 *     agent with more than CROWD_MAX_OBSTACLE_LINES segments in reach keeps
 *     the nearest ones and the call returns CROWD_EDEVICE, as crowd_step's
 *     next synchronising call would).
 *   - Device pointers: state_in [n][4] (px, py, vx, vy; the robot slot moves
 *     with the velocity stored there), state_out [n][4] (must not alias
 *     state_in), agent_params [n][4] (r, v_max, preferred speed, unused),
 *     goals [n][2], segments [n_segments][4] (zero-length segments are
 *     ignored).  Host pointers: box [4] (x0, y0, x1, y1), the region the grid
 *     covers, and p.  The box must contain every segment (CROWD_EINVAL
 *     otherwise); agents may leave it and are still handled exactly.
 *   - Results match crowd_step on a handle holding the same environment. */
#define CROWD_NOALLOC_MAX_AGENTS 65536
#define CROWD_NOALLOC_MAX_CELLS 65536
#define CROWD_NOALLOC_MAX_SEGMENT_CELLS (1 << 20)
crowd_status crowd_step_noalloc(int32_t n_agents, const float* state_in, float* state_out, const float* agent_params,
                                const float* goals, int32_t robot_index, int32_t n_segments, const float* segments,
                                const float* box, const crowd_params* p, float dt, void* cuda_stream);

/* ---- Occupancy-map front end (the step before the crowd step: the paper's
 * crowds live on generated maps of traversable ground and static objects,
 * with start and end points sampled on the traversable part, Sec. 3.1-3.2;
 * the raster form of such a map and these calls are this library's).
 *
 * occ: DEVICE [H][W] bytes, nonzero = obstacle; cell (x, y) covers
 * [x0 + x*cell, x0 + (x+1)*cell) x [y0 + y*cell, y0 + (y+1)*cell); W, H in
 * [1, 32768]; closed != 0: everything outside the map is obstacle (walls
 * round it), else free.  Coordinates are x0 + i*cell with the product and
 * the sum rounded to FP32 separately.  Both calls run on `stream`, allocate
 * and free temporary device memory, and wait for the stream before they
 * return.
 *
 * crowd_map_segments: the boundary between free and obstacle cells as
 * maximal axis-aligned segments [n][4] (ax, ay, bx, by) into DEVICE
 * `segments`, each directed with the free side on its left: horizontal lines
 * y = y0 + j*cell (j = 0..H) first, then vertical lines (i = 0..W), along each
 * line in increasing coordinate.  *n_segments gets the count; if it exceeds
 * max_segments nothing is written and CROWD_EINVAL is returned (call again
 * with a larger buffer). */
crowd_status crowd_map_segments(const uint8_t* occ, int32_t W, int32_t H, float cell, float x0, float y0,
                                int32_t closed, int32_t max_segments, float* segments, int32_t* n_segments,
                                void* stream);

/* Paper: Sec. 3.2 (random start and end points on the traversable area of
 * the occupancy map).
 * crowd_map_sample: n_points points [n][2] into DEVICE `points`, uniform over
 * the cells that are free and have no obstacle (and, when closed, no outside)
 * within `clearance` cells in x and y (0..CROWD_MAP_MAX_CLEARANCE).  Point k
 * draws (u0, u1, u2, u3) = Philox4x32-10(counter (k, stream_id, 0, 0), key
 * (seed low, seed high)); it lies in eligible cell floor(u0*M / 2^32) (M
 * eligible cells in row-major order) at fractions (u1 >> 8)/2^24 and
 * (u2 >> 8)/2^24 of the cell.  *n_eligible gets M; with n_points > 0 and
 * M = 0 the call fails with CROWD_EINVAL. */
#define CROWD_MAP_MAX_CLEARANCE 64
crowd_status crowd_map_sample(const uint8_t* occ, int32_t W, int32_t H, float cell, float x0, float y0,
                              int32_t closed, int32_t clearance, uint64_t seed, uint32_t stream_id, int32_t n_points,
                              float* points, int32_t* n_eligible, void* stream);

/* Message for the calling thread's last failed call ("" if none).
 * No counterpart in the paper (error reporting of this C interface). */
const char* crowd_last_error(void);

/* Library ABI version (increments on any signature change).
 * No counterpart in the paper. */
int32_t crowd_abi_version(void);  /* 5: crowd_read_launches, crowd_tuning.tiled_queue */

#ifdef __cplusplus
}
#endif

#endif /* CROWD_H */

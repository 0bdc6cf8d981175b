/*
 * ifem.h -- C ABI of libifem, the GB300 (sm_103a) implementation of the
 * immersed-finite-element (IFEM) fluid-structure coupling step of
 * Saadat, Guido, Iaccarino & Shaqfeh, "Immersed-finite-element method for
 * deformable particle suspensions in viscous and viscoelastic media"
 * (arXiv:1807.08219).
 *
 * The coupling step is the paper's Algorithm steps 1, 2 and 4:
 *   1. internal forces of every Lagrangian mesh (Eq. FEM for tetrahedral
 *      solids, Eq. FEM_Membrane plus the Helfrich bending force for
 *      triangulated membranes), summed per node;
 *   2. spreading of the nodal forces to the Eulerian grid, S*;
 *   4. interpolation of the grid velocity back to the nodes, S, with the
 *      same kernel.
 * The Navier-Stokes solve between 2 and 4 is not part of this library.
 *
 * ------------------------------------------------------------------------
 * Conventions shared by every entry point
 * ------------------------------------------------------------------------
 * Ownership. Handles (ifem_ctx, ifem_tmpl, ifem_grid, ifem_batch) own only
 *   their internal buffers. Every node and grid array passed to a compute
 *   call is caller-owned DEVICE memory (for example allocated by PyTorch);
 *   the library never frees, keeps or reallocates it. Host arrays passed to
 *   *_create functions are copied before the call returns.
 * Precision. A context computes in one precision (ifem_config.precision):
 *   IFEM_FP32: node and grid arrays are float; element kinematics, stress,
 *     spreading and interpolation run in FP32; reference-shape invariants
 *     (areas, volumes, inverse reference edge matrices) are derived in FP64
 *     on the host; conservation sums (ifem_reduce) are FP64.
 *   IFEM_FP64: node and grid arrays are double; deterministic: element
 *     forces, nodal sums, spreading and interpolation reproduce, bit for
 *     bit, the plain FP64 evaluation order documented with each operation
 *     (no fused multiply-add; nodal sums in ascending element order; each
 *     grid value summed over nodes in ascending node order). The bending
 *     force uses atan2 and is reproducible run to run, not bit-exact
 *     against other libm implementations.
 * Node arrays (x, F, v, w, Hw). Structure of arrays: 3 rows of N values,
 *   row a holding component a of every node: arr[a*N + k]. N is
 *   ifem_batch_nodes(batch); nodes of instance i are contiguous, instances
 *   in creation order, nodes in template order.
 * Positions. x holds each node's position RELATIVE to the FP64 origin of its
 *   instance (ifem_instance_desc.origin). Element forces depend on position
 *   differences only and are computed from these local values; the grid
 *   transfer uses origin + x. Keeping local offsets small keeps FP32 exact
 *   enough for edge vectors one grid cell long in a box of hundreds of
 *   cells.
 * Grid arrays (u, f). For every periodic box b of the grid, three staggered
 *   (MAC) lattices of n_b^3 values, one per velocity component d: lattice d
 *   has nodes at ((i, j, k) + o_d) h_b, o_d = (1/2,1/2,1/2) - e_d/2,
 *   h_b = L_b/n_b, stored x fastest: value (d, k, j, i) of box b at
 *   ifem_grid_box_offset(grid, b) + d*n_b^3 + (k*n_b + j)*n_b + i.
 * Streams. `stream` is a cudaStream_t (NULL = legacy default stream). Every
 *   compute call is asynchronous: its return value reports host-side
 *   argument checks and launch errors only. Errors found on the device
 *   (inverted elements, singular MLS moment matrices, capacity overflow,
 *   bounded-wait timeouts) are recorded in a device status block that
 *   ifem_sync_status() reads. No kernel traps.
 * Errors. Functions return ifem_status; IFEM_OK = 0, negative on error;
 *   ifem_last_error(ctx) gives a message for the last failed call on ctx.
 * Current device. A call that touches the GPU makes the context's device
 *   (ifem_config.device) current on the calling thread while it runs and
 *   restores the thread's previous current device before returning, so the
 *   caller's device selection is left as it was.
 */
#ifndef IFEM_H
#define IFEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ifem_ctx_s *ifem_ctx;     /* device state, workspace, status block */
typedef struct ifem_tmpl_s *ifem_tmpl;   /* one structure type: topology + reference data */
typedef struct ifem_grid_s *ifem_grid;   /* a set of periodic MAC boxes */
typedef struct ifem_batch_s *ifem_batch; /* particle instances of templates in boxes */

typedef enum {
    IFEM_OK = 0,
    IFEM_ERR_ARG = -1,       /* invalid argument (null handle, size, index, mismatch) */
    IFEM_ERR_OOM = -2,       /* device or host allocation failed */
    IFEM_ERR_CUDA = -3,      /* CUDA runtime error (message in ifem_last_error) */
    IFEM_ERR_TIMEOUT = -4,   /* a bounded device-side wait expired */
    IFEM_ERR_INVERTED = -5,  /* elements with J <= 0 were seen; forces still written */
    IFEM_ERR_DOMAIN = -6,    /* non-finite position or singular MLS moment matrix */
    IFEM_ERR_CAPACITY = -7   /* a size exceeds a documented library limit */
} ifem_status;

typedef enum { IFEM_FP32 = 0, IFEM_FP64 = 1 } ifem_precision;

/* Discrete delta kernels for S and S*.
 * PESKIN4: 4-point kernel of Peskin (2002), tensor product of
 *   phi(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4r^2))/8 for |r| <= 1,
 *            (5 - 2|r| - sqrt(-7 + 12|r| - 4r^2))/8 for 1 < |r| <= 2,
 *   r in cells, 4^3 lattice nodes per point.
 * MLS27: the paper's linear moving-least-squares kernel (Sec.
 *   "Interpolation Scheme"): the 27 lattice nodes around the nearest node,
 *   cubic-spline weight W(|x_J - x_k| / h_w), phi = p^T A^-1 B. */
typedef enum { IFEM_KERNEL_PESKIN4 = 0, IFEM_KERNEL_MLS27 = 1 } ifem_kernel;

/* Summation order of the FP32 scatters (IFEM_FP64 is always deterministic).
 * DET: forces are a fixed-order sum per node over its incident elements;
 * spreading sums each lattice value from the node lists of its own tile
 * (every node binned into each tile its stencil reaches), so repeated runs
 * give identical results.
 * ATOMIC: forces by atomic adds. With PESKIN4, spreading visits each node
 * once, in the tile holding its cell, accumulates into the tile plus a
 * 2-cell halo (4 in x) and adds that to the grid with atomic L2 adds, so the
 * order in which neighbouring tiles' halos combine is not reproducible. */
typedef enum { IFEM_SCATTER_DET = 0, IFEM_SCATTER_ATOMIC = 1 } ifem_scatter;

typedef enum { IFEM_LAW_NEO_HOOKE = 0, IFEM_LAW_SKALAK = 1 } ifem_membrane_law;

/* ifem_spread flags (bitwise or). */
#define IFEM_SPREAD_DENSITY 0   /* f_J += (n/L)^3 sum_k phi F_k (force per volume; default) */
#define IFEM_SPREAD_FORCE 1     /* f_J += sum_k phi F_k (the paper's literal nodal form) */
#define IFEM_SPREAD_OVERWRITE 2 /* f = 0 first over every box (dense), then add */

typedef struct {
    int precision;      /* ifem_precision */
    int kernel;         /* ifem_kernel */
    int scatter;        /* ifem_scatter */
    int tile;           /* node-bin tile edge in cells, 6..16; 0 = autotune in ifem_prepare */
    double mls_support; /* MLS weight radius h_w in cells; <= 0 means sqrt(3) */
    int device;         /* CUDA device ordinal the context is bound to */
    int profile;        /* 1: ifem_step_coupling records CUDA events around each stage */
} ifem_config;

/* Membrane constants. Neo-Hookean (Eq. neo-Hookena): W = mu/2 (I1 + 1/I2 - 3).
 * Skalak (Eq. Skalak): W = mu/2 (I1'^2/2 + I1' - I2') + C mu/8 I2'^2 with
 * I1' = I1 - 2, I2' = I2 - 1 (C = mu_D/mu). Helfrich bending modulus kb and
 * spontaneous curvature c0 (Eq. Bending_Energy); kb = 0 disables bending. */
typedef struct {
    double mu;
    double C;
    double kb;
    double c0;
} ifem_membrane_params;

/* Compressible neo-Hookean solid: W = lambda/4 (I3 - 1) - (lambda/2 + mu) ln I3^(1/2)
 * + mu/2 (I1 - 3) (Sec. Governing Equations). */
typedef struct {
    double lambda;
    double mu;
} ifem_solid_params;

typedef struct {
    int tmpl;          /* index into the template array given to ifem_batch_create */
    int box;           /* box index in the grid */
    double origin[3];  /* FP64 origin; node position = origin + x (box units) */
} ifem_instance_desc;

/* Device-side status, read back by ifem_sync_status. */
typedef struct {
    int64_t inverted_elements;  /* elements with J <= 0 in the last force evaluation */
    int64_t domain_errors;      /* non-finite positions / singular MLS matrices */
    int64_t capacity_errors;    /* per-tile list longer than the kernel's limit */
    int64_t timeouts;           /* bounded waits that expired */
    int64_t pairs;              /* (tile, node) pairs of the last binning (0 when the
                                   spread needs no per-tile candidate lists) */
    int64_t active_tiles;       /* tiles with at least one node pair */
    int64_t touched_cells;      /* non-zero lattice values added by spreads since the last sync
                                   (FP32 path; the FP64 path rewrites every value of an active
                                   tile; the FP32 ATOMIC Peskin spread counts the values inside
                                   each node's own tile only) */
} ifem_stats;

/* ---------------------------------------------------------------- context */
/* Fill cfg with defaults: FP32, PESKIN4, DET scatter, tile 0 (auto), device 0. */
int ifem_config_default(ifem_config *cfg);
/* Create a context bound to cfg->device. Allocates the device status block. */
int ifem_ctx_create(const ifem_config *cfg, ifem_ctx *out);
int ifem_ctx_destroy(ifem_ctx ctx);
/* Message of the last failed call on ctx (never NULL; "" if none). */
const char *ifem_last_error(ifem_ctx ctx);
/* Wait for the context's last stream, copy the status block to *out and reset
 * it. Returns the most severe recorded device error (IFEM_ERR_TIMEOUT,
 * IFEM_ERR_DOMAIN, IFEM_ERR_CAPACITY, IFEM_ERR_INVERTED) or IFEM_OK. */
int ifem_sync_status(ifem_ctx ctx, ifem_stats *out);
/* Tile edge (cells) currently used by ctx (after autotuning, if any). */
int ifem_ctx_tile(ifem_ctx ctx);
/* Stage durations of the last ifem_step_coupling(_ab2, _host) call on a context created
 * with cfg.profile = 1, measured with CUDA events recorded on that call's
 * stream: ms[0] binning, ms[1] forces, ms[2] spread, ms[3] interpolation,
 * ms[4] reductions (milliseconds); where the step fuses interpolation into
 * the spread (see ifem_step_coupling) ms[2] covers both and ms[3] is 0.
 * Waits for the last recorded event.
 * IFEM_ERR_ARG if profiling is off or no step has run. */
int ifem_stage_times(ifem_ctx ctx, double *ms);

/* -------------------------------------------------------------- templates */
/* Triangulated membrane (Eq. FEM_Membrane). tris: host int32 (n_tris, 3),
 * oriented with (b-a)x(c-a) pointing outward; X_ref: host double (n_nodes, 3)
 * AoS, the stress-free configuration. Reference data per triangle (in-plane
 * inverse edge matrix, area A0) is derived in FP64 here. The surface must be
 * a closed 2-manifold when kb != 0. IFEM_FP32 contexts accept up to 8192
 * nodes per template (IFEM_ERR_CAPACITY beyond). */
int ifem_tmpl_create_membrane(ifem_ctx ctx, int n_nodes, int n_tris, const int32_t *tris,
                              const double *X_ref, int law, const ifem_membrane_params *p,
                              ifem_tmpl *out);
/* Tetrahedral solid (Eq. FEM). tets: host int32 (n_tets, 4) with
 * det[X1-X0, X2-X0, X3-X0] > 0 (IFEM_ERR_ARG otherwise); X_ref as above.
 * Reference gradients of the shape functions and V0 derived in FP64 here. */
int ifem_tmpl_create_solid(ifem_ctx ctx, int n_nodes, int n_tets, const int32_t *tets,
                           const double *X_ref, const ifem_solid_params *p, ifem_tmpl *out);
int ifem_tmpl_destroy(ifem_tmpl t);

/* ------------------------------------------------------------------- grid */
/* n_boxes periodic boxes; n: host int32 cells per side (8..1024), L: host
 * double side lengths (> 0). */
int ifem_grid_create(ifem_ctx ctx, int n_boxes, const int32_t *n, const double *L, ifem_grid *out);
int ifem_grid_destroy(ifem_grid g);
/* Total number of values of one grid field (sum over boxes of 3 n_b^3). */
int64_t ifem_grid_values(ifem_grid g);
/* Offset of box b's first value within a grid field. */
int64_t ifem_grid_box_offset(ifem_grid g, int b);

/* ------------------------------------------------------------------ batch */
/* Instances of the given templates placed in the boxes of `grid`. The batch
 * keeps references to the templates and the grid: destroy it first. */
int ifem_batch_create(ifem_ctx ctx, int n_tmpl, const ifem_tmpl *tmpls, int n_inst,
                      const ifem_instance_desc *inst, ifem_grid grid, ifem_batch *out);
int ifem_batch_destroy(ifem_batch b);
int64_t ifem_batch_nodes(ifem_batch b);
int ifem_batch_instances(ifem_batch b);
/* Replace the instance origins (host double, 3 per instance). */
int ifem_batch_set_origins(ifem_batch b, const double *origins);
/* Allocate every work buffer that the compute calls on (ctx, b) need, so
 * that later calls allocate nothing (for example inside CUDA-graph capture).
 * If ctx was created with tile = 0 and has not been tuned yet, first run the
 * tile autotuner: binning + spreading + interpolation of b at positions x
 * (device node array, required then) are timed with CUDA events on `stream`
 * for tile edges {8, 12, 16} (FP32) or {6, 8, 10} (FP64), and the fastest is
 * kept (ifem_ctx_tile). Autotuning allocates temporary buffers and
 * synchronises: call it outside stream capture. Without ifem_prepare, a
 * context with tile = 0 uses 16 (FP32) or 8 (FP64). */
int ifem_prepare(ifem_ctx ctx, ifem_batch b, const void *x, void *stream);

/* --------------------------------------------------------------- compute */
/* Algorithm step 1: internal nodal forces F = F_el + F_be (membranes) or
 * F_el (solids) of every instance, F = -dE/dx for the elastic part:
 *   membranes: F_k = -A0 P^ grad N^_k, P^ = F^ S^, S^ = 2 dW/dC^ (Eq. FEM_Membrane);
 *   solids:    F_k = -V0 P grad N_k, P = F S,
 *              S = lambda/2 (J^2 - 1) C^-1 + mu (I - C^-1) (Eq. FEM);
 *   bending:   F_k = 2 kb [Lap_s(kH - kH0) + 2 (kH - kH0)(kH^2 - kG + kH0 kH)] n_k A_k
 *              with kH0 = -c0/2 and the cotangent / mixed-Voronoi operators of
 *              Meyer, Desbrun, Schroeder & Barr (2003).
 * x: device node array (local positions); F: device node array, overwritten.
 * Elements with J <= 0 still contribute and are counted in the status block. */
int ifem_compute_forces(ifem_ctx ctx, ifem_batch b, const void *x, void *F, void *stream);

/* Algorithm step 2, spreading S*: for every lattice value J of the boxes,
 *   f_J += s sum_k phi(x_J - (origin_k + x_k)) F_k,  s = (n_b/L_b)^3 (density)
 *   or 1 (IFEM_SPREAD_FORCE), summed over the nodes k of the instances in
 *   that box; periodic wrap. x, F: device node arrays; f: device grid field.
 * IFEM_FP64 evaluation order per value: f = f + w*g over nodes in ascending
 * order, g = F_k,d * s, w = (phi_x*phi_y)*phi_z (PESKIN4). */
int ifem_spread(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, const void *F,
                void *f, int flags, void *stream);

/* Algorithm step 4, interpolation S: v_k,d = sum_J phi(x_J - (origin_k + x_k)) u_J,d.
 * u: device grid field; x: device node array; v: device node array,
 * overwritten. IFEM_FP64 order: from 0, stencil z-outer, x-inner,
 * acc = acc + w*u. */
int ifem_interpolate(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *u, const void *x,
                     void *v, void *stream);

/* Interpolation S (Sec. "Interpolation Scheme") of a cell-centred field with
 * ncomp components, e.g. the six components of the polymer conformation
 * tensor C_J that the fluid-stress forces of solids need:
 *   out_k,q = sum_J phi(x_J - (origin_k + x_k)) field_J,q,  x_J = ((i,j,k) + 1/2) h_b.
 * field: device array, box b holding ncomp blocks of n_b^3 values (x fastest)
 * from value offset (ifem_grid_box_offset(g, b) / 3) * ncomp; x: device node
 * array; out: device array of ncomp rows of N (row q = component q), overwritten.
 * ncomp in 1..64. Kernel and precision as the context; IFEM_FP64 order per
 * node and component: acc = acc + w*c from 0, stencil z-outer, x-inner. */
int ifem_interpolate_cc(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *field, int ncomp,
                        const void *x, void *out, void *stream);

/* Fluid properties for the fluid-stress forces inside solids: solvent +
 * polymer viscosity eta, viscosity ratio beta, polymer relaxation time lambda
 * (Sec. "Governing Equations"). */
typedef struct {
    double eta;
    double beta;
    double lambda;
} ifem_fluid_params;

/* ifem_fluid_stress_forces flags */
#define IFEM_FORCES_ACCUMULATE 1 /* F = F + fluid forces (default: F overwritten) */

/* Fluid-stress parts of the immersed-boundary force inside solid particles
 * (Sec. "Governing Equations" and Eq. FEM with P^s - P^{f,N} - P^{f,P}):
 *   F^N_k + F^P_k = V0 (P^{f,N} + P^{f,P}) grad N_k per tet, summed over tets,
 *   P^{f,N} = eta J (grad u + grad u^T) F^-T,  grad u = sum_k u_k (x) grad N_k F^-1,
 *   P^{f,P} = J eta (1 - beta)/lambda (sum_k (C_k - I)/4) F^-T.
 * x: device node array (local positions); u: device node array of node
 * velocities (e.g. from ifem_interpolate); C: device array of 6 rows of N
 * (xx, yy, zz, xy, xz, yz, e.g. from ifem_interpolate_cc) or NULL for no
 * polymer term; F: device node array, overwritten (or accumulated into with
 * IFEM_FORCES_ACCUMULATE). Membrane nodes receive 0 (no fluid stress in the
 * thin-shell model). Deterministic in both precisions (per-element buffer,
 * then a fixed-order nodal sum); IFEM_FP64 follows the evaluation order
 * written beside the kernel. IFEM_ERR_ARG for eta < 0 or, with C, lambda <= 0. */
int ifem_fluid_stress_forces(ifem_ctx ctx, ifem_batch b, const void *x, const void *u, const void *C,
                             const ifem_fluid_params *p, void *F, int flags, void *stream);

/* Source of the indicator-function equation lap I = div G of the variable-
 * viscosity model (Sec. "Variable Viscosity Implementation"):
 *   G_J = s sum_k n_k A_k phi(x_J - (origin_k + x_k)),
 * n_k A_k the unit vertex normal times the mixed Voronoi area of membrane
 * node k (the operators of the bending force; solid nodes contribute 0),
 * spread onto the three MAC lattices exactly as ifem_spread spreads a force:
 * same kernels, flags, precision and summation order (s = (n_b/L_b)^3, or 1
 * with IFEM_SPREAD_FORCE). x: device node array; G: device grid field. Uses
 * the batch's internal scratch: calls on one batch must not overlap on the
 * GPU. The Poisson solve itself is not part of this library. */
int ifem_indicator_source(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, void *G, int flags,
                          void *stream);

/* ------------------------------------------------------ Lagrangian update */
/* Adams-Bashforth position update (Eq. Bashforth_eqn), in place:
 *   x = x + dt (3/2 v - 1/2 v_prev)
 * x, v, v_prev: device node arrays (x: the particles' local positions).
 * Both precisions evaluate x + dt*(1.5*v - 0.5*v_prev) in that order, one
 * rounding per operation (no fused multiply-adds). For the
 * first step pass v_prev = v (forward Euler). IFEM_ERR_ARG for a non-finite dt. */
int ifem_ab2_update(ifem_ctx ctx, ifem_batch b, void *x, const void *v, const void *v_prev, double dt,
                    void *stream);

/* Current volume of every particle, FP64 in both precisions: membranes by the
 * polyhedron formula of Sec. "Conservation of Volume for Membranes",
 *   V = 1/18 sum_faces [x1.(x2 x x3) + x2.(x3 x x1) + x3.(x1 x x2)],
 * solids as the sum of their tets' signed volumes det(Ds)/6. x: device node
 * array; vol: device double array of n_inst, overwritten. Fixed-order block
 * sums: reproducible run to run. */
int ifem_volumes(ifem_ctx ctx, ifem_batch b, const void *x, double *vol, void *stream);

/* Membrane volume correction (Sec. "Conservation of Volume for Membranes",
 * after Mendez et al. 2014), in place: x_I = x_I + Lambda alpha_I with
 *   alpha_I = -(1/12) sum over the faces containing I of x_I2 x x_I3 (the
 *             face's other two nodes in cyclic order),
 * Lambda the root, reached by Newton's method from 0, of
 *   A L^3 + B L^2 + C L + D = 0, A = 1/18 sum alpha.(alpha x alpha),
 *   B = 1/6 sum x.(alpha x alpha), C = 1/6 sum alpha.(x x x) (all cyclic over
 *   each face's nodes), D = V(x) - V0.
 * The cubic's sums and Lambda are FP64 in both precisions; with IFEM_FP32
 * positions alpha comes from FP32 cross products of the ring's edge vectors
 * (equal to the formula above on a closed ring), and since the cubic is built
 * from that same alpha the corrected volume still meets V0. V0: device double array of n_inst
 * target volumes; lambda: device double array of n_inst receiving Lambda
 * (0 for solids, which are left unchanged), or NULL. An instance whose Newton
 * iteration does not converge in 100 steps is left unchanged and counted in
 * domain_errors. Uses the batch's internal scratch: calls on one batch must
 * not overlap on the GPU. */
int ifem_volume_correct(ifem_ctx ctx, ifem_batch b, void *x, const double *V0, double *lambda, void *stream);

/* FP64 conservation sums per instance i (ifem_reduce layout, 12 doubles):
 *   [0..2]  centroid c_i = mean of the local positions x_k
 *   [3..5]  sum_k F_k
 *   [6..8]  sum_k (x_k - c_i) x F_k      (torque about the centroid)
 *   [9..11] sum_k v_k
 * then 6 doubles per box b: [0..2] h_b^3 sum_J f_J,d of the values the last
 * spread ADDED in box b, [3..5] reserved (0). Sums are FP64 in a fixed order
 * (block trees), reproducible run to run. red: device double array of
 * 12*n_inst + 6*n_boxes. F or v may be NULL (their entries are then 0). */
int ifem_reduce(ifem_ctx ctx, ifem_batch b, const void *x, const void *F, const void *v,
                double *red, void *stream);

/* The whole coupling step in one call: bin, forces -> F, spread F -> f
 * (flags as ifem_spread), interpolate u -> v, reductions -> red (may be
 * NULL). Gives the results of the four calls above. The forces run beside
 * the binning and the interpolation beside the spreading, on two streams the
 * context owns, forked from `stream` with events and joined back into it
 * before the reductions (valid under CUDA-graph capture of `stream`); with
 * cfg.profile = 1 the stages run one after the other on `stream` instead
 * (forces, then binning, spreading, interpolation, reductions), so that
 * ifem_stage_times can attribute them. With IFEM_FP32, IFEM_SCATTER_ATOMIC
 * and IFEM_KERNEL_PESKIN4 the interpolation is fused into the spreading
 * kernel (each node's stencil weights serve both transfers), and the last
 * part of the binning waits for the forces: it also sums |F| per tile, which
 * sets the spread accumulators' fixed-point scales. Results equal those of
 * the separate calls up to FP32 rounding. */
int ifem_step_coupling(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, const void *u,
                       void *F, void *f, void *v, double *red, int flags, void *stream);

/* The coupling step followed by the position update of Algorithm step 4 and
 * Eq. Bashforth_eqn, out of place:
 *   x_new = x + dt (3/2 v - 1/2 v_prev)
 * with v the velocities this step interpolates. Arguments as
 * ifem_step_coupling, plus v_prev (device node array, the previous step's
 * velocities; pass v_prev = a copy of v for a forward-Euler first step) and
 * x_new (device node array receiving the new local positions). Where the
 * step fuses the interpolation into the spreading kernel (IFEM_FP32,
 * IFEM_SCATTER_ATOMIC, IFEM_KERNEL_PESKIN4) the same kernel also writes x_new
 * from each velocity it gathers, so v is never read back; elsewhere the update
 * runs after the interpolation on its stream. x_new equals ifem_ab2_update on
 * a copy of x with the v this call writes (bit for bit). x_new may not overlap
 * x, v, v_prev or F, nor v_prev overlap v (IFEM_ERR_ARG); IFEM_ERR_ARG for a
 * non-finite dt. */
int ifem_step_coupling_ab2(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x, const void *u,
                           void *F, void *f, void *v, double *red, int flags, const void *v_prev,
                           double dt, void *x_new, void *stream);

/* The coupling step for a caller whose node arrays live in host memory (a
 * fluid solver on the CPU, the paper's Algorithm steps 1, 2 and 4 with the
 * exchange of x and v in the loop): x_host (3 x N, the context's real type,
 * the layout of x) is copied into the device work array x, the step runs as
 * ifem_step_coupling on x, u, F, f, v, red, and v is copied back into v_host
 * (3 x N) and, when red_host is given, the sums into red_host (12*n_inst +
 * 6*n_boxes doubles; needs red). All copies are asynchronous on `stream`
 * and the context's auxiliary streams, joined back into `stream`: the host
 * arrays must stay valid, and v_host and red_host are filled, only once
 * `stream` has passed this point. Host arrays should be pinned
 * (cudaHostAlloc); pageable memory works outside graph capture but copies
 * without overlap. With IFEM_FP32, IFEM_SCATTER_ATOMIC and a batch of two or
 * more particles the positions arrive in two halves (by particle) and each
 * half's element forces start as soon as it has landed; with the Peskin
 * kernel the fused spreading and interpolation then run as one launch per
 * lattice, and row d of v goes back to the host as soon as lattice d is done
 * (rows 0 and 1 beside the later lattices, row 2 beside the sums of v and the
 * boxes); lattices 1 and 2 are launched with programmatic serialization, so
 * that their blocks start as the previous lattice's run out of work (within
 * stream capture this becomes a programmatic edge of the graph). Results
 * equal those of copying x in, calling
 * ifem_step_coupling and copying v and red out. Returns IFEM_ERR_ARG for null
 * host arrays (N > 0) or red_host without red. */
int ifem_step_coupling_host(ifem_ctx ctx, ifem_batch b, ifem_grid g, const void *x_host, void *x,
                            const void *u, void *F, void *f, void *v, void *v_host, double *red,
                            double *red_host, int flags, void *stream);

/* Hessian-vector product of the elastic energy (bending excluded):
 *   Hw = d/de [-F_el(x + e w)] at e = 0,
 * by the analytic directional derivative of the element stresses. w, Hw:
 * device node arrays; Hw overwritten. Used for the adjoint of
 * ifem_compute_forces: (dF/dx)^T g = -H g (H symmetric). */
int ifem_force_hvp(ifem_ctx ctx, ifem_batch b, const void *x, const void *w, void *Hw, void *stream);

/* ifem_compute_forces without any allocation in the call. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate.
 * Some callers of this library cannot call cudaMalloc: hosts that hand all
 * device memory to their own pool or allocator at start-up (a second
 * allocator fails or fragments their memory), and real-time loops that forbid
 * allocation once running (cudaMalloc may synchronise the device and takes
 * unbounded time). This entry point computes the forces of
 * ifem_compute_forces through the deterministic element-buffer path
 * (per-element forces, then a per-node sum in ascending element order, then
 * the bending passes), taking its scratch from one fixed array of 32 MiB in
 * device memory that the library declares at file scope: every GPU that
 * loads libifem holds it until the process exits. It calls no cudaMalloc,
 * cudaFree or allocating library routine. The caller still passes x and F.
 *   Limit: 12 reals per element plus 6 reals per node (reals of the
 *   context's precision; the node part starts at a 256-byte boundary) must
 *   fit in 32 MiB, e.g. about 600k triangles in IFEM_FP32; larger batches
 *   are rejected with IFEM_ERR_CAPACITY before anything is launched.
 *   Set-up: the first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Sharing: every call on a device uses the same array, which keeps the
 *   last call's contents; each call writes every entry it later reads, so
 *   nothing needs clearing. Calls whose kernels overlap on the GPU (other
 *   streams, other threads) race on the array: serialise them.
 * Arguments, layouts, stream semantics and status reporting are those of
 * ifem_compute_forces; the FP32 results are deterministic but may differ in
 * the last bits from ifem_compute_forces (this path uses no fused
 * multiply-add). Launch errors are reported for the first launch that failed;
 * no kernel after it is queued. */
int ifem_compute_forces_noalloc(ifem_ctx ctx, ifem_batch b, const void *x, void *F, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* IFEM_H */

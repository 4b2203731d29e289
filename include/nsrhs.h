/*
 * nsrhs — element-by-element assembly of the incompressible Navier-Stokes
 * right-hand side on linear tetrahedra, on one NVIDIA GB300 (sm_103a).
 *
 * What is assembled (the paper, arXiv 2403.08777, names the method but prints
 * no formulas; this is the library's definition of it):
 *   - the RHS of the explicit momentum step of an incompressible LES
 *     (Sec. II), plus the continuity residual, on linear tets with 4 nodes and
 *     4 Gauss points and constant shape-function gradients (Sec. V-B);
 *   - constant density rho and viscosity mu; Vreman eddy viscosity computed
 *     once per element from the constant velocity gradient (Sec. V-B);
 *   - SUPG/PSPG stabilisation, tau = 1/(c1 mu_eff/h^2 + c2 rho |u|/h) at each
 *     Gauss point, h = detJ^(1/3);
 *   - the element RHS computed directly, without element matrices (Sec. V-A),
 *     and scatter-added into the global nodal RHS (Sec. V-D).
 *   For test function N_a of an element (u, p linear on it):
 *     F_a,i = int[ -rho N_a (u.grad)u_i - mu_eff grad N_a.grad u_i + p dN_a/dx_i
 *                  - tau rho (u.grad N_a)(rho (u.grad)u_i + dp/dx_i) ]
 *     F_a,4 = int[ -N_a div u - tau grad N_a.(rho (u.grad)u + grad p) ]
 *   with every integral evaluated by the 4-point degree-2 rule, and
 *   RHS[conn[a][e]] += F_a over all elements e and local nodes a.
 *
 * Layouts (structure of arrays, node or element index fastest):
 *   coords [3][n_nodes] double        x, y, z
 *   conn   [4][n_elems] int32         local node a of element e at conn[a*n_elems + e]
 *   up     [4][n_nodes] double/float  u, v, w, p
 *   rhs, cot, grad [4][n_nodes] double
 *
 * Execution: every call is asynchronous on the CUDA stream it is given
 * (NULL = legacy default stream) except nsrhs_mesh_create, which
 * synchronises that stream once to read back its validation result.
 * Device pointers only (cudaMalloc, cudaMallocAsync, managed memory, or
 * torch CUDA tensors). A kernel fault surfaces as NSRHS_ECUDA on the call
 * that launched it or on a later call.
 *
 * Errors: no call throws. On NSRHS_EINVAL the outputs are untouched. Status
 * strings come from nsrhs_status_string.
 */
#ifndef NSRHS_H
#define NSRHS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nsrhs_mesh nsrhs_mesh; /* opaque; owned by the library */

typedef enum {
  NSRHS_OK = 0,
  NSRHS_EINVAL = 1,      /* bad argument: NULL pointer, size <= 0 or too large,
                            unknown enum value, destroyed mesh */
  NSRHS_ENOMEM = 2,      /* device allocation failed */
  NSRHS_EMESH = 3,       /* connectivity index out of [0, n_nodes) or an element
                            with detJ <= 0 (no silent reorientation) */
  NSRHS_ECUDA = 4,       /* a CUDA runtime call or kernel launch failed */
  NSRHS_EUNSUPPORTED = 5 /* valid request that this build does not implement */
} nsrhs_status;

typedef enum {
  NSRHS_FP64 = 0, /* double precision throughout */
  NSRHS_MIXED = 1 /* float nodal (u,p) and float element arithmetic (with
                     the hardware's approximate reciprocal and square roots);
                     the element geometry (det and inverse) computed in double
                     once per mesh for every element, so also for those whose
                     aspect ratio exceeds the mesh's threshold, then rounded;
                     double global accumulation */
} nsrhs_precision;

typedef enum {
  NSRHS_SCATTER_AUTO = 0,   /* the measured fastest for the precision */
  NSRHS_SCATTER_ATOMIC = 1, /* one double-precision atomic add per entry */
  NSRHS_SCATTER_BLOCK = 2,  /* per-block node-local accumulation in shared
                               memory, one atomic per (block, node, component);
                               forward and adjoint. The shared-memory stages
                               are sized by the mesh's largest block (its
                               distinct nodes); where the FP64 adjoint's stages
                               cannot fit one CTA (with 227 KB per CTA, a block
                               of 256 elements touching more than 672 distinct
                               nodes, 576 for the one-pass call, e.g.
                               disconnected elements), that call returns
                               NSRHS_EUNSUPPORTED */
  NSRHS_SCATTER_COLOUR = 3, /* element colouring: elements sharing a node have
                               different colours; one launch per colour, whose
                               atomic adds never meet at one address, so the
                               summation order is fixed and results are
                               bitwise reproducible. Needs a mesh created with
                               opts.colour = 1, else NSRHS_EUNSUPPORTED */
  NSRHS_SCATTER_BLOCK_COLOUR = 4 /* BLOCK with its blocks coloured (blocks
                               sharing a node differ): per-block node sums in a
                               fixed order, then one launch per block colour;
                               bitwise reproducible; forward and adjoint.
                               Needs opts.colour = 1 */
} nsrhs_scatter;

typedef enum {
  NSRHS_CONVECTIVE = 0, /* Galerkin convection -rho int N_a (u.grad)u_i */
  NSRHS_SKEW = 1        /* skew-symmetric -rho/2 int [N_a (u.grad)u_i - (u.grad N_a) u_i]:
                           the convective RHS does no work on the discrete
                           velocity (the energy-preserving property of Sec. II) */
} nsrhs_convection;

typedef enum {
  NSRHS_TAU_GAUSS = 0,  /* tau at each Gauss point from |u_g| */
  NSRHS_TAU_ELEMENT = 1 /* one tau per element from |mean nodal velocity| */
} nsrhs_tau_mode;

typedef enum {
  NSRHS_GEOM_CACHED = 0,   /* read each element's cofactors, 1/detJ and
                              detJ^(-1/3), computed in double once per mesh
                              (88 bytes per element streamed per call) */
  NSRHS_GEOM_RECOMPUTE = 1 /* form the Jacobian, its cofactors, 1/detJ and
                              detJ^(-1/3) from the gathered node coordinates in
                              every call (Sec. V-B: constant shape-function
                              gradients per element): 43 more FP64 operations
                              per element instead of the streamed record.
                              NSRHS_FP64 with scatter AUTO or ATOMIC, in
                              nsrhs_assemble and nsrhs_assemble_vjp only;
                              otherwise NSRHS_EUNSUPPORTED */
} nsrhs_geometry;

/* Physical and numerical parameters (uniform over one call). */
typedef struct {
  double rho;         /* density, >= 0 */
  double mu;          /* dynamic viscosity, > 0 */
  double c_vreman;    /* Vreman constant (about 0.07); 0 switches the model off */
  double c1, c2;      /* stabilisation constants of tau (4 and 2) */
  int32_t precision;  /* nsrhs_precision */
  int32_t scatter;    /* nsrhs_scatter */
  int32_t convection; /* nsrhs_convection */
  int32_t tau_mode;   /* nsrhs_tau_mode */
  int32_t geometry;   /* nsrhs_geometry */
  int32_t reserved;   /* must be 0 */
} nsrhs_params;

/* Mesh options. */
typedef struct {
  double ar_threshold; /* aspect ratio above which an element counts as high-AR
                          in nsrhs_mesh_info.n_high_ar; 10 by default.
                          AR = l_max S / (6 sqrt(6) V) (l_max longest edge,
                          S surface, V volume; 1 for the regular tet). The
                          threshold changes no arithmetic: the geometry of
                          every element is computed in double once per mesh
                          (and rounded to float for the mixed form). */
  int32_t colour;      /* 1: also colour the elements and keep a colour-major
                          copy of the connectivity and geometry (about 150
                          bytes per element more) for NSRHS_SCATTER_COLOUR,
                          and colour the element blocks for
                          NSRHS_SCATTER_BLOCK_COLOUR; 0 (default): not.
                          Greedy colouring, at most 128 colours, else mesh
                          creation returns NSRHS_EUNSUPPORTED. */
  int32_t reserved;    /* must be 0 */
} nsrhs_mesh_opts;

/* Read-only facts about a created mesh. */
typedef struct {
  int64_t n_nodes, n_elems;
  int64_t n_high_ar;      /* elements with AR > ar_threshold */
  int64_t n_blocks;       /* element blocks of the BLOCK scatter */
  int64_t block_elems;    /* elements per block */
  int64_t device_bytes;   /* device memory held by the mesh */
  double min_detj, max_ar;
  int64_t n_colours;      /* colours of the COLOUR scatter; 0 if not built */
  int64_t n_block_colours; /* block colours of BLOCK_COLOUR; 0 if not built */
} nsrhs_mesh_info;

/* Fill *p with rho=1, mu=1e-2, c_vreman=0, c1=4, c2=2, FP64, AUTO,
   convective form, tau at the Gauss points, cached geometry. */
void nsrhs_params_default(nsrhs_params* p);

/* Fill *o with ar_threshold = 10, colour = 0. */
void nsrhs_mesh_opts_default(nsrhs_mesh_opts* o);

/*
 * Create a mesh from device arrays coords [3][n_nodes] and conn [4][n_elems].
 * The library copies both (the caller may free them afterwards), checks on
 * the device that every index is in range and every element has detJ > 0,
 * classifies elements by aspect ratio, orders them along a Morton curve of
 * their centroids, caches their geometry, and builds the element blocks of
 * the BLOCK scatter (and, with opts->colour, the colourings of the COLOUR
 * and BLOCK_COLOUR scatters). opts may be NULL (defaults). Synchronises
 * `stream` (with colouring, once per colouring round).
 * 1 <= n_nodes < 2^31, 1 <= n_elems < 2^31.
 * On error *out is set to NULL and nothing is leaked.
 */
nsrhs_status nsrhs_mesh_create(int64_t n_nodes, int64_t n_elems, const double* coords,
                               const int32_t* conn, const nsrhs_mesh_opts* opts, void* stream,
                               nsrhs_mesh** out);

nsrhs_status nsrhs_mesh_get_info(const nsrhs_mesh* m, nsrhs_mesh_info* info);

/*
 * rhs = assembled RHS of (up) on mesh m (see the definition above).
 * up is [4][n_nodes] double for NSRHS_FP64 and [4][n_nodes] float for
 * NSRHS_MIXED; rhs [4][n_nodes] double is overwritten (zeroed, then summed
 * into). up and rhs must not overlap. The summation order of the atomic
 * adds is unspecified, so results agree with a serial sum to rounding only;
 * with NSRHS_SCATTER_COLOUR and NSRHS_SCATTER_BLOCK_COLOUR the order is
 * fixed and repeated calls give bitwise identical results.
 */
nsrhs_status nsrhs_assemble(const nsrhs_mesh* m, const nsrhs_params* p, const void* up,
                            double* rhs, void* stream);

/*
 * Vector-Jacobian product of the assembly: grad = (d rhs / d up)^T cot,
 * the adjoint of nsrhs_assemble with respect to the nodal velocity and
 * pressure (the mesh and parameters are constants). NSRHS_FP64: up and cot
 * [4][n_nodes] double. NSRHS_MIXED: up and cot [4][n_nodes] float, float
 * reverse sweep, double accumulation. grad [4][n_nodes] double is
 * overwritten. The element quantities are recomputed, not stored. Where a
 * Gauss-point velocity is exactly zero, |u_g| contributes the symmetric
 * derivative 0. Scatter modes as for nsrhs_assemble.
 */
nsrhs_status nsrhs_assemble_vjp(const nsrhs_mesh* m, const nsrhs_params* p, const void* up,
                                const void* cot, double* grad, void* stream);

/*
 * Both of the above at the same state in one pass: rhs = assembled RHS of up
 * and grad = (d rhs / d up)^T cot, with one gather of up and cot per element
 * and the element's forward intermediates computed once (the adjoint's
 * recomputation of them is shared with the RHS). For callers that hold the
 * cotangent before the RHS is needed: residual and adjoint-residual sweeps
 * of steady adjoint solvers, one-shot optimisation, Newton-Krylov with a
 * transposed product. Types and layouts as nsrhs_assemble / _vjp; rhs and
 * grad must be distinct and are overwritten. Scatter AUTO (atomics for
 * NSRHS_FP64, blocks for NSRHS_MIXED), ATOMIC, BLOCK or BLOCK_COLOUR (the
 * block stages hold the cotangent beside (u, p) and two entry buffers, the
 * element RHS and its gradient, summed per node by the same runs;
 * NSRHS_EUNSUPPORTED where they do not fit a CTA's shared memory, as for the
 * FP64 adjoint). NSRHS_SCATTER_COLOUR, NSRHS_GEOM_RECOMPUTE, and
 * BLOCK_COLOUR on a mesh created without colouring: NSRHS_EUNSUPPORTED.
 * A null pointer, a destroyed or foreign mesh, or rhs == grad: NSRHS_EINVAL.
 * On either error nothing is written.
 */
nsrhs_status nsrhs_assemble_rhs_vjp(const nsrhs_mesh* m, const nsrhs_params* p, const void* up,
                                    const void* cot, double* rhs, double* grad, void* stream);

/*
 * The same RHS (FP64, convective form, tau at the Gauss points) computed the
 * way the paper's baseline did before its restructuring (Sec. V-A): with the
 * nonlinear coefficients frozen at the current state, a full 16x16 element
 * matrix per tet, multiplied by the element unknowns. A comparison path that
 * measures the gain of the direct form; rhs is overwritten. Other precisions
 * or variants: NSRHS_EUNSUPPORTED.
 */
nsrhs_status nsrhs_assemble_elmat(const nsrhs_mesh* m, const nsrhs_params* p, const double* up,
                                  double* rhs, void* stream);

/*
 * ---- Explicit time stepping of the momentum equation ----
 * The paper's kernel is the RHS of an explicit momentum step (Sec. II); these
 * calls take that step. With the row-sum lumped P1 mass
 *   m_a = sum over the elements containing node a of V_e / 4,
 * the semi-discrete momentum equation is rho m_a du_a/dt = F_a (the first
 * three rows of the assembled RHS). The pressure is held fixed (its
 * fractional-step solve is outside this library).
 */
typedef enum {
  NSRHS_EULER = 0, /* u' = u + dt L(u) */
  NSRHS_SSPRK3 = 1 /* Shu-Osher three-stage strong-stability-preserving Runge-Kutta:
                      u1 = u + dt L(u); u2 = 3/4 u + 1/4 (u1 + dt L(u1));
                      u' = 1/3 u + 2/3 (u2 + dt L(u2)) */
} nsrhs_time_scheme;

/* Lumped mass of every node into mass_dev [n_nodes] double (overwritten). */
nsrhs_status nsrhs_lumped_mass(const nsrhs_mesh* m, double* mass_dev, void* stream);

/*
 * One explicit step of length dt > 0 with L(u) = F(u, p) / (rho m), on
 * up_dev [4][n_nodes] double in place (rows u, v, w advanced, row p kept).
 * work_dev: caller-owned device scratch (no allocation inside) of
 * 8 * n_nodes doubles for NSRHS_FP64, 10 * n_nodes for NSRHS_MIXED (which
 * assembles each stage's RHS from a float copy of the double state, with
 * float element arithmetic and double accumulation; the state and its
 * update stay double). Requires rho > 0. Each Runge-Kutta stage runs one
 * nsrhs_assemble on the stream.
 */
nsrhs_status nsrhs_explicit_step(const nsrhs_mesh* m, const nsrhs_params* p, double dt,
                                 int32_t scheme, double* up_dev, double* work_dev, void* stream);

/*
 * Per element, in the caller's element order, into out_dev [n_elems] int32
 * (device memory, overwritten):
 *   NSRHS_ELEMENT_COLOUR        its colour in the COLOUR scatter, 0 .. n_colours - 1
 *                               (two elements that share a node never have the
 *                               same colour);
 *   NSRHS_ELEMENT_BLOCK_COLOUR  the colour of its block in the BLOCK_COLOUR
 *                               scatter, 0 .. n_block_colours - 1 (elements of
 *                               two different blocks of the same colour never
 *                               share a node);
 *   NSRHS_ELEMENT_BLOCK         the index of its block.
 * Only for a mesh created with opts.colour = 1, else NSRHS_EUNSUPPORTED;
 * another `which`: NSRHS_EINVAL. For checking and inspection.
 */
typedef enum {
  NSRHS_ELEMENT_COLOUR = 0,
  NSRHS_ELEMENT_BLOCK_COLOUR = 1,
  NSRHS_ELEMENT_BLOCK = 2
} nsrhs_element_property;

nsrhs_status nsrhs_mesh_element_colours(const nsrhs_mesh* m, int32_t which, int32_t* out_dev,
                                        void* stream);

/* Free the mesh and its device memory. NULL-safe. Synchronises the device
   memory it frees (cudaFree semantics). */
void nsrhs_destroy(nsrhs_mesh* m);

const char* nsrhs_status_string(nsrhs_status s);

/*
 * ---- Mesh check that allocates nothing ----
 * The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory: code that owns all GPU memory through its
 * own fixed arena, or runs where a cudaMalloc (which may synchronise the
 * device, fail late, or be forbidden by the host framework) is not allowed.
 * nsrhs_mesh_create copies the mesh and allocates scratch for its checks;
 * this call performs the same checks on the caller's arrays in place and
 * writes only to the caller's result.
 *
 * Checks every element of coords [3][n_nodes] / conn [4][n_elems] (device
 * arrays) exactly as nsrhs_mesh_create does and writes one
 * nsrhs_mesh_check_result into *result_dev (caller-owned DEVICE memory):
 * the number of elements with an index out of [0, n_nodes), the number with
 * detJ <= 0, the number with aspect ratio > ar_threshold, and the minimum
 * detJ / maximum aspect ratio over the valid elements (+inf / 0 if none).
 * Asynchronous on `stream`; read the result after synchronising it.
 *
 * Scratch: a file-scope device array of NSRHS_CHECK_SCRATCH_BLOCKS partial
 * results (64 bytes each, 64 KiB in all) that every GPU which loads the
 * library holds until the process exits. Every call writes the partials it
 * uses before reading them, so no state carries over from the last call; but
 * all calls share that one array, so calls whose kernels overlap on the GPU
 * (different streams, or different host threads, without ordering between
 * them) race and may return wrong results. Serialise them.
 *
 * The first call on each device looks up the array's device address (with
 * that device current) and remembers it; make that first call before any
 * stream capture. 1 <= n_nodes, n_elems < 2^31 and ar_threshold > 0, else
 * NSRHS_EINVAL. No cudaMalloc, cudaFree or other allocating call is made.
 */
#define NSRHS_CHECK_SCRATCH_BLOCKS 1024

typedef struct {
  int64_t bad_index; /* elements with a node index outside [0, n_nodes) */
  int64_t bad_det;   /* elements with detJ <= 0 */
  int64_t n_high_ar; /* valid elements with aspect ratio > ar_threshold */
  double min_detj;   /* over valid elements */
  double max_ar;     /* over valid elements */
} nsrhs_mesh_check_result;

nsrhs_status nsrhs_mesh_check_noalloc(int64_t n_nodes, int64_t n_elems, const double* coords,
                                      const int32_t* conn, double ar_threshold, void* stream,
                                      nsrhs_mesh_check_result* result_dev);

#ifdef __cplusplus
}
#endif

#endif /* NSRHS_H */

/*
 * gipc.h -- C ABI of the GB300 Gauss-Newton IPC hot path.
 *
 * The library evaluates the rewritten simplicial-measure contact barrier of
 * Huang et al., "GIPC: Fast and stable Gauss-Newton optimization of IPC
 * barrier energy" (the paper), its gradient and its analytically PSD-projected
 * Hessian per contact stencil, and the pieces of the Gauss-Newton step that
 * consume them.
 *
 * Conventions shared by every call
 *  - Pointers are DEVICE pointers unless the name ends in `_h` (host).
 *  - The caller owns every input and output buffer.  A context owns only its
 *    own scratch memory.
 *  - Every call enqueues its work on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream), returns without synchronising unless its comment
 *    says otherwise, and never calls cudaDeviceSynchronize.
 *  - Positions are float64 structure-of-arrays: x[0*n + i], x[1*n + i],
 *    x[2*n + i] are the x, y, z coordinates of vertex i.
 *  - Per-stencil outputs are "entry-major": entry j of stencil i is stored at
 *    out[j*k + i], so one warp writes 32 consecutive values of one entry.
 *  - Every call returns a gipc_status.  On failure gipc_last_error() gives a
 *    message (per host thread).  Arguments are checked on the host before
 *    any launch; a call that fails its checks enqueues nothing.
 */
#ifndef GIPC_H
#define GIPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GIPC_OK = 0,
    GIPC_ERR_INVALID_ARG = -1,   /* a pointer, size or option failed the host checks   */
    GIPC_ERR_CUDA = -2,          /* a CUDA runtime call or kernel launch failed          */
    GIPC_ERR_OOM = -3,           /* device scratch could not be allocated                */
    GIPC_ERR_NOT_CONVERGED = -4, /* an iteration cap was reached                         */
    GIPC_ERR_NONFINITE = -5,     /* a NaN or Inf was detected in device data             */
    GIPC_ERR_TIMEOUT = -6,       /* a bounded device wait expired                        */
    GIPC_ERR_CAPACITY = -7,      /* an output buffer is smaller than the result          */
    GIPC_ERR_INDEFINITE = -8     /* the solver met c . H c <= 0: H is not positive definite
                                  * on the free coordinates (the last iterate is returned) */
} gipc_status;

/* Contact stencil types.  The type is carried by the signs of the stencil's
 * four vertex indices (paper Sec. 7.2, "Data structures"):
 *   EE [+,+,+,+]  PT [-,+,+,+]  PE [-,+,+,#]  PP [-,+,#,#]
 *   nearly parallel: EE [+,-,+,+]  PE [-,-,+,-]  PP [-,-,-,-]
 * A negative slot stores -(i+1) (= ~i), so vertex 0 can carry a sign; '#'
 * is GIPC_NULL_INDEX.  Vertex slot order after decoding:
 *   PT      point, triangle v0, v1, v2
 *   EE      edge-a end 0, edge-a end 1, edge-b end 0, edge-b end 1
 *   PE      point, edge end 0, edge end 1
 *   PP      point a, point b
 *   EE_PAR  as EE
 *   PE_PAR  point, other end of the point's edge, edge end 0, edge end 1
 *   PP_PAR  point a, other end of a's edge, point b, other end of b's edge
 * The distance of PE_PAR is between slots 0 and (2,3); of PP_PAR between
 * slots 0 and 2; the parallel measure c always uses the edges (0,1), (2,3). */
typedef enum {
    GIPC_PT = 0, GIPC_EE = 1, GIPC_PE = 2, GIPC_PP = 3,
    GIPC_EE_PAR = 4, GIPC_PE_PAR = 5, GIPC_PP_PAR = 6
} gipc_stencil_type;

#define GIPC_NULL_INDEX ((int32_t)(-2147483647 - 1))

/* Per-stencil flag bits written by gipc_eval_stencils. */
#define GIPC_FLAG_ACTIVE    0x01u   /* d < dhat: the barrier is non-zero                    */
#define GIPC_FLAG_FILTERED  0x02u   /* g < eps_g: Eq. 23 replaced lambda_1 by lambda_1^thr  */
#define GIPC_FLAG_MOLLIFIED 0x04u   /* c < eps_x: the mollifier of Eq. 25 is active         */
#define GIPC_FLAG_INVALID   0x80u   /* malformed tuple or index >= n: energy/lam 0, rest unwritten */

typedef enum { GIPC_FP64 = 0, GIPC_MIXED = 1 } gipc_precision;

typedef enum {
    GIPC_HESS_DENSE = 0,   /* the full 3s x 3s block per stencil                        */
    GIPC_HESS_RANK1 = 1,   /* (lambda, w) with block = lambda * w w^T                    */
    GIPC_HESS_BLOCKS = 2   /* the same dense values, element-major as 16 contiguous 3x3
                            * sub-blocks: entry (3a+i, 3b+j) of element e at
                            * [(e * 16 + 4a + b) * 9 + 3i + j] ([count][16][9]; the
                            * sub-blocks of slots >= s are not written, except that
                            * gipc_eval_stencils may set to zero the first entry of
                            * such a sub-block that directly follows a written one)  */
} gipc_hess_mode;

/* Parameters of the barrier (paper Sec. 5.3-5.4, 6.1).  Lengths are in the
 * units of the positions. */
typedef struct {
    double dhat;          /* computational accuracy target d-hat (> 0)                   */
    double kappa;         /* barrier stiffness multiplying every stencil energy (>= 0)   */
    double d_thr_ratio;   /* d_thr / dhat of the proximal filter (paper: 0.1), in (0,1)  */
} gipc_barrier_params;

typedef struct gipc_ctx gipc_ctx;

/* Create / destroy a context.  A context holds scratch for the calls that need
 * it and binds to the device that is current at creation. */
gipc_status gipc_create(gipc_ctx** ctx_out_h);
gipc_status gipc_destroy(gipc_ctx* ctx);

/* Message of the last failure on the calling host thread ("" if none). */
const char* gipc_last_error(void);

/* eps_x of the nearly-parallel mollifier (paper Sec. 6.1, below Eq. 25):
 *   eps_x = 1e-3 * ||xbar_{12} - xbar_{11}||^2 * ||xbar_{22} - xbar_{21}||^2
 * from REST positions `rest_x` ([3][n] float64) for the two edges of every
 * EE-derived stencil (slots (0,1) and (2,3)); 0 for PT, PE and PP.
 *   stencils   int32 [4][k], sign-encoded (see gipc_stencil_type)
 *   eps_x_out  float64 [k]
 * Malformed tuples or indices >= n give eps_x = 0 (no read out of range).
 * Errors: GIPC_ERR_INVALID_ARG for n < 0, k < 0 or a null pointer with k > 0. */
gipc_status gipc_compute_eps_x(const double* rest_x, int64_t n, const int32_t* stencils,
                               int64_t k, double* eps_x_out, void* stream);

/* Barrier energy, gradient and PSD-projected Hessian of every stencil
 * (paper Alg. 2 per pair; Eq. 7-36).
 *
 * For each stencil with vertices x_s (s = 2, 3 or 4):
 *   g = d^2 / dhat^2 with d the distance of its type (Eq. 4-5, Eq. 9-11);
 *   inactive (all outputs 0, flags 0) when g >= 1;
 *   b(g) = dhat^4 (1-g)^2 ln^2 g (Eq. 24), energy = kappa * b;
 *   plain types:   grad = kappa * b_g * dg/dx,
 *                  H = kappa * lambda1_hat * w w^T with w = df/dx, f = sqrt(g),
 *                  lambda1 = 4 g b_gg + 2 b_g (Eq. 18), replaced by its value at
 *                  g = eps_g = d_thr_ratio^2 when g < eps_g (Eq. 23);
 *   parallel types: btilde = e(c) b(g) with the mollifier of Eq. 25 (c the
 *                  parallel measure, eps_x as given), grad = kappa * dbtilde/dx,
 *                  H = kappa * lambda8' * w w^T (Eq. 36) with
 *                  w = q0 * dsqrt(c)/dx + q1 * df/dx, (q0, q1) the unit
 *                  eigenvector of [[lambda_gamma1, 4t], [4t, lambda_g1]] for its
 *                  larger eigenvalue lambda8' (Eq. 33-35), q1 >= 0.  The filter of
 *                  Eq. 23 is applied to lambda_g1.
 * Geometry (distances, cross products, the parallel measure) is evaluated with
 * error-free transformations in double-double precision, so g and c are
 * correctly rounded float64 values except in rare rounding ties.
 *
 * Arguments
 *   x          float64 [3][n] positions
 *   stencils   int32 [4][k] sign-encoded tuples
 *   eps_x      float64 [k] (from gipc_compute_eps_x); may be NULL when the list
 *              holds no parallel types (then eps_x = 0: mollifier inactive)
 *   prm_h      barrier parameters (host)
 *   prec       GIPC_FP64, or GIPC_MIXED (Hessian blocks / w written as float32)
 *   mode       GIPC_HESS_DENSE, GIPC_HESS_BLOCKS or GIPC_HESS_RANK1
 *   energy     float64 [k] or NULL
 *   grad       float64 [12][k] or NULL; entries j < 3s used (slot-major x,y,z)
 *   hess       DENSE: [144][k] entries a*3s+b for a, b < 3s (row-major block);
 *              BLOCKS: [k][16][9], the same values as 3x3 sub-blocks (see the enum);
 *              RANK1: [12][k] holding w (entries j < 3s);
 *              float64 for GIPC_FP64, float32 for GIPC_MIXED; or NULL
 *   lam        float64 [k] (RANK1 only; kappa * lambda) or NULL
 *   flags      uint8 [k] (GIPC_FLAG_*) or NULL
 * Entries beyond a stencil's 3s (or (3s)^2) are not written, nor are the
 * gradient / Hessian entries of an invalid stencil (GIPC_FLAG_INVALID).
 * Errors: GIPC_ERR_INVALID_ARG (bad sizes, null x/stencils with k > 0,
 * dhat <= 0, kappa < 0, d_thr_ratio outside (0,1), unknown prec/mode),
 * GIPC_ERR_CUDA (launch failure). */
gipc_status gipc_eval_stencils(const double* x, int64_t n, const int32_t* stencils, int64_t k,
                               const double* eps_x, const gipc_barrier_params* prm_h,
                               int prec, int mode, double* energy, double* grad, void* hess,
                               double* lam, uint8_t* flags, void* stream);

/* ------------------------------------------------------------------ tetrahedra */

/* Stable neo-Hookean parameters: Psi = mu/2 (I2 - 3) + lambda/2 (J - alpha)^2
 * - mu/2 log(I2 + 1), alpha = 1 + mu/lambda - mu/(4 lambda) (paper Sec. 8: the
 * deformables use the Stable neo-Hookean energy). */
typedef struct {
    double mu, lambda;   /* energy parameters (from gipc_snh_params)                     */
    double scale;        /* multiplies energy, gradient and Hessian (dt^2 in the step)    */
} gipc_elastic_params;

/* (mu, lambda) of the energy above from Young's modulus and Poisson's ratio:
 * mu = 4/3 mu_L, lambda = lambda_L + 5/6 mu_L with the Lame parameters of (E, nu),
 * so small strains behave as linear elasticity with (mu_L, lambda_L).  Host only. */
gipc_status gipc_snh_params(double young, double poisson, double* mu_h, double* lambda_h);

/* Rest state of tetrahedra from rest positions (float64 [3][n]):
 *   Dm_inv  float64 [9][T]: inverse of Dm = [xbar1-xbar0, xbar2-xbar0, xbar3-xbar0], row-major
 *   vol     float64 [T]:    |det Dm| / 6
 *   mass    float64 [n] or NULL: lumped masses density * sum(vol)/4 over incident tetrahedra,
 *           summed in ascending tetrahedron index (reproducible bit for bit)
 * tets: int32 [4][T] vertex ids.  Synchronises the stream once (to report degenerate
 * elements).  Errors: GIPC_ERR_INVALID_ARG (sizes, pointers, a zero-volume or
 * out-of-range tetrahedron), GIPC_ERR_OOM, GIPC_ERR_CUDA. */
gipc_status gipc_tet_rest(gipc_ctx* ctx, const double* rest_x, int64_t n, const int32_t* tets, int64_t T,
                          double density, double* Dm_inv, double* vol, double* mass, void* stream);

/* Energy scale*vol*Psi(F), gradient and PSD-projected Hessian of every tetrahedron,
 * F = Ds Dm^-1.  The projection uses the closed-form eigensystem of the isotropic energy
 * (twist, flip and scaling modes from a rotation-variant SVD of F), keeping the modes
 * with positive eigenvalues.
 *   energy float64 [T] or NULL; grad float64 [12][T] or NULL;
 *   hess_mode  GIPC_HESS_DENSE: hess [144][T] (row-major 12x12, vertex-major x,y,z);
 *              GIPC_HESS_BLOCKS: hess [T][16][9] (3x3 sub-blocks, see the enum)
 *   hess   float64 (GIPC_FP64), or float32 (GIPC_MIXED: the projection computed in float32
 *          arithmetic; energy and gradient stay float64), or NULL
 * A tetrahedron with a vertex id outside [0, n) gets energy 0 and no other output.
 * Errors: GIPC_ERR_INVALID_ARG, GIPC_ERR_CUDA. */
gipc_status gipc_eval_tets(const double* x, int64_t n, const int32_t* tets, int64_t T, const double* Dm_inv,
                           const double* vol, const gipc_elastic_params* prm_h, int prec, int hess_mode,
                           double* energy, double* grad, void* hess, void* stream);

/* ------------------------------------------------------------------ assembly */

/* A square 3x3-block sparse matrix (BSR) over n block rows.  Block p of row r
 * (rowptr[r] <= p < rowptr[r+1]) sits at block column colidx[p], columns
 * ascending within a row; its 9 values are vals[9p + 3i + j] (row-major). */
typedef struct {
    int64_t n;         /* block rows (= vertices); set by gipc_assemble_bsr      */
    int64_t nnzb;      /* stored blocks; set by gipc_assemble_bsr                */
    int64_t capacity;  /* capacity of colidx / vals in blocks (caller)           */
    int32_t* rowptr;   /* [n+1]                                                  */
    int32_t* colidx;   /* [capacity]                                             */
    void* vals;        /* [capacity][9]: float64 (GIPC_FP64) or float32 (GIPC_MIXED) */
    int prec;          /* GIPC_FP64 or GIPC_MIXED (caller)                       */
} gipc_bsr;

/* One list of elements with their local blocks, in the layout
 * gipc_eval_stencils (stencils) or gipc_eval_tets (tetrahedra) writes. */
typedef struct {
    const int32_t* idx;   /* stencils: int32 [4][count] sign-encoded; tets: int32 [4][count] vertex ids */
    int64_t count;
    int hess_mode;        /* GIPC_HESS_DENSE ([144][count]), GIPC_HESS_BLOCKS ([count][16][9]) or,
                           * stencils only, GIPC_HESS_RANK1                                         */
    const void* hess;     /* dense blocks or w [12][count]; float64 / float32 as the BSR's prec     */
    const double* lam;    /* RANK1: lambda [count] (block = lam * w w^T)                              */
    const double* grad;   /* float64 [12][count] element gradients, or NULL                          */
} gipc_elements;

/* Assemble H = M + sum_e P_e^T H_e P_e into `bsr` and, if grad_out is given,
 * g = grad_base + sum_e P_e^T g_e into grad_out (float64 [3][n]).
 * (Paper: the Newton system of Alg. 1, lines "g <- dI/dx" and
 * "H <- M + getPSDForceJacobian(...)"; the local-to-global decomposition of
 * the system matrix in supplement Sec. S6.)
 *
 * Pattern: every ordered vertex pair of every element plus (i, i) for each
 * vertex when `mass` is given, built by a key sort; identical on every run.
 * Values: each block sums, in this order, m_i I_3 (diagonal, if mass), then
 * the sub-blocks of its tetrahedra in ascending index, then those of its
 * stencils in ascending index -- a fixed order, so results are reproducible
 * bit for bit.  Elements that are malformed or reference a vertex >= n are
 * skipped.  `stencils_h` / `tets_h` (host structs) may be NULL.
 *
 *   mass       float64 [n] lumped vertex masses, or NULL (no diagonal terms)
 *   grad_base  float64 [3][n] added first to the gradient (e.g. inertia), or NULL
 *
 * Blocks until the pattern size is known (one stream synchronisation), then
 * enqueues the value pass.  Scratch is owned by ctx and reused across calls.
 * Errors: GIPC_ERR_INVALID_ARG; GIPC_ERR_CAPACITY when nnzb > bsr->capacity
 * (bsr->nnzb then holds the required count and rowptr is valid) or nnzb does
 * not fit int32; GIPC_ERR_OOM; GIPC_ERR_CUDA. */
gipc_status gipc_assemble_bsr(gipc_ctx* ctx, int64_t n, const gipc_elements* stencils_h,
                              const gipc_elements* tets_h, const double* mass, const double* grad_base,
                              gipc_bsr* bsr_h, double* grad_out, void* stream);

/* ------------------------------------------------------------------ solver */

/* Arithmetic of the matrix-vector product H c inside the solver (FP64 matrices; ignored for
 * GIPC_MIXED matrices, batched solves and gipc_pcg_noalloc, which use the native form). */
typedef enum {
    GIPC_PRODUCT_NATIVE = 0,      /* FP64 products and sums                                          */
    GIPC_PRODUCT_FLOAT_PAIR = 1   /* each FP64 value of H and c split once into two float32 (x = hi +
                                   * lo), products and sums in double-float arithmetic (Dekker's exact
                                   * product, Knuth's TwoSum) on the FP32 pipe, the row result rounded to
                                   * FP64: about 2^-44 relative per row instead of 2^-52, the same bytes,
                                   * a fraction of the FP64 instructions.  Values below ~1e-30 in
                                   * magnitude lose their low part (float32 range).                    */
} gipc_product;

typedef struct {
    double rel_tol;    /* stop when delta_new < rel_tol * delta_0 (paper Sec. 8: 1e-4); 0 runs max_iter */
    int max_iter;      /* iteration cap (>= 0)                                                        */
    int check_every;   /* host checks for convergence every this many iterations; 0 = automatic       */
    int product;       /* gipc_product of H c (0: native)                                              */
    int flags;         /* 0, or GIPC_PCG_STOP_ON_INDEFINITE                                             */
} gipc_pcg_params;

/* gipc_pcg_params.flags: stop with GIPC_ERR_INDEFINITE when a search direction has c . H c <= 0
 * (one system; ignored by batched solves).  Off by default: the paper's modified PCG continues,
 * and near its rounding floor a float32 product can give c . H c <= 0 for a positive definite H. */
#define GIPC_PCG_STOP_ON_INDEFINITE 1

/* Solve H x = rhs by modified PCG with a 3x3 block-Jacobi preconditioner
 * (paper Sec. 7.2 "Parallel solver optimizations" and "Preconditioning of the
 * CG solver"; termination delta_new < rel_tol * delta_0 from Sec. 8).
 *
 *   r = S(rhs - H x0), z = P^-1 r, c = S(z), delta_0 = r.z; then per iteration
 *   q = S(H c), alpha = delta/(c.q), x += alpha c, r -= alpha q, s = P^-1 r,
 *   delta' = r.s, c = S(s + (delta'/delta) c)
 * with P = blockdiag(H_ii) (identity where a diagonal block is missing or not
 * positive definite) and S zeroing the vertices with fixed[i] != 0 ("modified"
 * PCG).  P^-1 is applied through a per-vertex LDL^T factorisation, so r.z is a
 * sum of squares and stays nonnegative on very ill-conditioned blocks.
 *
 *   A      BSR matrix (n = A->n block rows); FP64 or float32 values (MIXED: the
 *          products and row sums are float32, and so are the block-Jacobi factors,
 *          s = P^-1 r and the direction c, whose exact float64 image updates x and
 *          enters the dots; x, r, alpha, beta and the dots are float64)
 *   rhs    float64 [3][n]
 *   x      float64 [3][n]: initial guess in, solution out (fixed vertices: 0)
 *   fixed  uint8 [n] or NULL
 *   iters_out_h, rel_out_h  (host, may be NULL) iterations run, delta_new/delta_0
 * Dot products are reduced in a fixed order: identical inputs give identical
 * results.  Synchronises the stream at the end (and every check_every
 * iterations when rel_tol > 0).
 * Errors: GIPC_ERR_INVALID_ARG; GIPC_ERR_NOT_CONVERGED (rel_tol > 0 and the cap
 * was reached; x holds the last iterate); GIPC_ERR_INDEFINITE (with
 * GIPC_PCG_STOP_ON_INDEFINITE: c . H c <= 0 for a search direction, H is not positive
 * definite on the free coordinates; x holds the last iterate); GIPC_ERR_NONFINITE;
 * GIPC_ERR_OOM; GIPC_ERR_CUDA. */
gipc_status gipc_pcg(gipc_ctx* ctx, const gipc_bsr* A_h, const double* rhs, double* x,
                     const uint8_t* fixed, const gipc_pcg_params* prm_h, int* iters_out_h,
                     double* rel_out_h, void* stream);

/* Largest system (block rows) gipc_pcg_noalloc accepts. */
#define GIPC_PCG_NOALLOC_MAX_N 32768

/* gipc_pcg without a context and without any device allocation.  (The paper
 * has no counterpart: this entry point exists for callers, not for the method.)
 *
 * For callers that may not allocate device memory -- for example a host
 * framework that owns all device memory through its own pool and forbids
 * cudaMalloc, or a latency-critical loop in which cudaMalloc/cudaFree (which
 * can synchronise the device) would stall work on other streams.  It runs the
 * same algorithm as gipc_pcg with the same arguments and results, with the
 * matrix product taken row by row from the BSR arrays (no sliced copy of the
 * matrix, no persistent launch), and keeps its working vectors in one fixed
 * array of about 7.2 MB in device global memory that the library defines:
 * every GPU that loads the library holds that array until the process exits.
 * The caller still passes the matrix, rhs and x.  prm_h->product must be
 * GIPC_PRODUCT_NATIVE or GIPC_PRODUCT_FLOAT_PAIR; both run the native FP64
 * product here.
 *
 *  - Limit: A->n <= GIPC_PCG_NOALLOC_MAX_N; larger systems are rejected with
 *    GIPC_ERR_INVALID_ARG and a message naming the limit (nothing is enqueued).
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any
 *    stream capture.
 *  - Like gipc_pcg, the call waits for its stream at the end (and every
 *    check_every iterations when rel_tol > 0) to read the iteration count and
 *    the status.
 *  - All calls share the one array, which keeps the last call's contents; each
 *    call clears what must start at zero (the solver's counters and flags).
 *    Calls that overlap on the GPU (e.g. issued on two streams at once, or from
 *    two host threads) race on the array and give wrong results: serialise them.
 * Errors and outputs as gipc_pcg. */
gipc_status gipc_pcg_noalloc(const gipc_bsr* A_h, const double* rhs, double* x, const uint8_t* fixed,
                             const gipc_pcg_params* prm_h, int* iters_out_h, double* rel_out_h,
                             void* stream);

/* ------------------------------------------------------------------ contacts */

/* The collision surface: device arrays of vertex ids, each in [0, n) (not
 * checked on the device). */
typedef struct {
    const int32_t* tris;   /* int32 [3][ntri] surface triangles                        */
    int64_t ntri;
    const int32_t* edges;  /* int32 [2][nedge] surface edges                            */
    int64_t nedge;
    const int32_t* verts;  /* int32 [nvert] surface vertices                            */
    int64_t nvert;
} gipc_surface;

/* The contact stencils of the barrier at positions x (paper Eq. 3 over the
 * point-triangle pairs of Eq. 4 and the edge-edge pairs of Eq. 5).
 *
 * A pair is a surface vertex and a surface triangle not containing it, or two
 * surface edges i < j without a shared vertex.  Every pair whose distance is
 * below dhat yields one stencil, typed by the closest features of its
 * constrained minimum (interior, point-edge or point-point; Sec. 3.1) and
 * encoded as in Sec. 7.2.  Edge-edge pairs whose parallel measure
 * c = |(a1-a0) x (b1-b0)|^2 is below eps_x (Sec. 6.1, computed from rest_x)
 * take the nearly-parallel types.  Pairs are screened by bounding boxes padded
 * by dhat (1 + 1e-9); the distance test and classification are float64 IEEE
 * operations in a fixed order without contraction.
 *
 *   x, rest_x  float64 [3][n]
 *   stencils   int32 [4][capacity] out: the first *count_h columns
 *   eps_x      float64 [capacity] out: 0 for point-triangle pairs,
 *              1e-3 |a1-a0|^2 |b1-b0|^2 at rest for edge-edge pairs
 *   count_h    host out: number of contacts
 * Order: point-triangle pairs by (surface-vertex position in verts, triangle),
 * then edge-edge pairs by (i, j); identical on every run.  Synchronises the
 * stream once (to read the count).  Errors: GIPC_ERR_INVALID_ARG;
 * GIPC_ERR_CAPACITY when *count_h > capacity (nothing is written; *count_h
 * holds the required size); GIPC_ERR_OOM; GIPC_ERR_CUDA. */
gipc_status gipc_find_contacts(gipc_ctx* ctx, const double* x, const double* rest_x, int64_t n,
                               const gipc_surface* srf_h, double dhat, int32_t* stencils, double* eps_x,
                               int64_t capacity, int64_t* count_h, void* stream);

/* Largest feasible step along d (paper Alg. 1, "maxFeasibleStepSize"):
 * alpha = min(1, min over pairs of the additive-CCD time of the motion x -> x + d).
 * Every point-triangle and edge-edge pair (as in gipc_find_contacts) whose swept
 * bounding boxes overlap is advanced conservatively with its common translation
 * removed: first step (1 - slack) d0 / l_p, then 0.9 d / l_p, stopping once the
 * distance falls below slack * d0 (d0 the initial distance, l_p the bound on
 * the relative motion).  Result in [0, 1] on the host.  Synchronises the stream.
 *   x, d   float64 [3][n];  slack in (0, 1) (0.1 is the usual value)
 * Errors: GIPC_ERR_INVALID_ARG; GIPC_ERR_OOM; GIPC_ERR_CUDA. */
gipc_status gipc_ccd_max_step(gipc_ctx* ctx, const double* x, const double* d, int64_t n,
                              const gipc_surface* srf_h, double slack, double* alpha_h, void* stream);

/* ------------------------------------------------------------------ time step */

/* A simulated scene: tetrahedral meshes, their surface and the fixed vertices.
 * All arrays are device arrays the caller keeps alive during a step. */
typedef struct {
    int64_t n;                /* vertices                                               */
    const double* rest_x;     /* float64 [3][n] rest positions (eps_x of edge pairs)    */
    const int32_t* tets;      /* int32 [4][T]                                           */
    int64_t T;
    const double* Dm_inv;     /* float64 [9][T] from gipc_tet_rest                      */
    const double* vol;        /* float64 [T]                                            */
    const double* mass;       /* float64 [n] lumped masses                              */
    const uint8_t* fixed;     /* uint8 [n] (nonzero: prescribed, kept in place) or NULL */
    gipc_surface surface;
    double l;                 /* length of the scene's bounding-box diagonal            */
} gipc_scene;

typedef struct {
    double dt;               /* time step                                                    */
    double gravity[3];       /* body acceleration                                            */
    gipc_elastic_params elastic;  /* scale is ignored (dt^2 is used)                         */
    gipc_barrier_params barrier;
    double eps_d;            /* stop when max|d| / (l dt) <= eps_d                           */
    double pcg_tol;          /* gipc_pcg_params.rel_tol of each Newton solve                 */
    int max_pcg;             /* PCG iteration cap per Newton iteration                       */
    int max_newton;          /* Newton iteration cap                                         */
    int max_ls;              /* line-search trials per Newton iteration                      */
    int prec;                /* GIPC_FP64 or GIPC_MIXED (Hessian storage and SpMV)           */
    int hess_mode;           /* GIPC_HESS_DENSE or GIPC_HESS_RANK1 for the contact stencils  */
} gipc_step_params;

typedef struct {
    int newton_iters;        /* Newton iterations taken                                     */
    int pcg_iters;           /* PCG iterations summed over the Newton iterations            */
    int ls_trials;           /* line-search energy evaluations summed                       */
    int converged;           /* 1 if the eps_d test ended the loop                          */
    int64_t contacts;        /* contact stencils at the final positions                     */
    double energy;           /* incremental potential at the final positions                */
    double last_alpha;       /* step length of the last Newton iteration                    */
} gipc_step_stats;

/* One implicit time step by projected Newton (paper Alg. 1) on the incremental
 * potential (Sec. 3.1, Eq. 1-2):
 *   I(x) = 1/2 (x - xt)^T M (x - xt) + dt^2 sum_T vol Psi(F) + kappa sum_k b_k(x),
 *   xt = x^t + dt v^t + dt^2 gravity (fixed vertices: xt = x^t).
 * Each iteration: contacts at x; g and H = M + PSD-projected Hessians assembled
 * into a BSR matrix; d from the modified PCG (fixed vertices filtered; a solve
 * that reaches max_pcg is used as it is); alpha = gipc_ccd_max_step(x, d, 0.1);
 * backtracking alpha /= 2 until I(x + alpha d) <= I(x), contacts re-detected at
 * each trial (after max_ls trials the last one is kept); stop when
 * max|d| / (l dt) <= eps_d or after max_newton iterations.
 *   x  float64 [3][n]: x^t in, x^{t+1} out
 *   v  float64 [3][n]: v^t in, (x^{t+1} - x^t) / dt out
 * Synchronises the stream several times per iteration.  Scratch is owned by ctx.
 * Errors: GIPC_ERR_INVALID_ARG; GIPC_ERR_NONFINITE; GIPC_ERR_OOM; GIPC_ERR_CUDA;
 * GIPC_ERR_CAPACITY (more than 2^31 matrix blocks). */
gipc_status gipc_newton_step(gipc_ctx* ctx, const gipc_scene* sc_h, double* x, double* v,
                             const gipc_step_params* prm_h, gipc_step_stats* stats_h, void* stream);

/* Many independent scenes advanced together (batched time step).  The paper has no batched
 * form; this is the batching extension of the hot path.
 *
 * `all` is the concatenation of the scenes: scene k owns the vertices
 * [vert_off_h[k], vert_off_h[k+1]); every tetrahedron, surface triangle, edge and vertex lies in
 * one scene, and the tetrahedra and the three surface lists are ordered by scene.  all.l is not
 * used (l_h gives each scene's bounding-box diagonal for its stopping test). */
typedef struct {
    gipc_scene all;
    int32_t nscenes;
    const int64_t* vert_off_h;   /* [nscenes+1] host, from 0 to all.n, strictly increasing */
    const double* l_h;           /* [nscenes] host */
} gipc_scene_batch;

/* One implicit time step of every scene (the Newton loop of gipc_newton_step per scene), all
 * scenes in one set of launches per phase: contacts are never formed across scenes (the broad
 * phase keys its cells by scene), the system matrix is block diagonal, the PCG keeps each
 * scene's own alpha, beta, residual and stopping test, and the CCD step, line-search step,
 * incremental potential and Newton stopping test are per scene.  A scene whose test is met stops
 * moving while the others continue.
 *   x, v      as gipc_newton_step, over all vertices
 *   stats_h   [nscenes] per-scene statistics (host), or NULL
 * Errors: as gipc_newton_step; GIPC_ERR_INVALID_ARG also when an element spans two scenes or a
 * list is not ordered by scene (checked on the device, one synchronisation). */
gipc_status gipc_newton_step_batch(gipc_ctx* ctx, const gipc_scene_batch* batch_h, double* x, double* v,
                                   const gipc_step_params* prm_h, gipc_step_stats* stats_h, void* stream);

/* ------------------------------------------------------------------ differentiation */
/* The paper has no derivatives with respect to the simulation inputs; this section is the
 * differentiation extension of the hot path.  Everything here is EXACT (no PSD projection):
 * element energies are evaluated with hyper-dual numbers, so gradients, Hessian-vector products
 * and Hessian blocks carry no truncation error. */

/* out = base + sum_e P_e^T v_e: element vectors v_e (the `grad` field of each list, [12][count]
 * slot-major as gipc_eval_* write them) summed per vertex in ascending element order (tetrahedra
 * first), the order of the assembled gradient.  `hess`, `lam` and `hess_mode` are ignored.
 *   base  float64 [3][n] or NULL;  out  float64 [3][n]
 * Never synchronises.  Errors: GIPC_ERR_INVALID_ARG, GIPC_ERR_OOM, GIPC_ERR_CUDA. */
gipc_status gipc_scatter_elements(gipc_ctx* ctx, int64_t n, const gipc_elements* stencils_h,
                                  const gipc_elements* tets_h, const double* base, double* out, void* stream);

/* The incremental potential at x for a given contact list (stencils [4][k], eps_x [k]):
 *   I(x) = 1/2 (x - xt)^T M (x - xt) + ep.scale sum_T vol Psi(F) + sum_k kappa btilde_k(x)
 * (Sec. 3.1, Eq. 1-2, Eq. 24-25; Psi as gipc_eval_tets, btilde as gipc_eval_stencils' energy) and
 * its exact derivatives:
 *   energy_h  host scalar or NULL (synchronises when given)
 *   grad      float64 [3][n] or NULL:  dI/dx
 *   Hu        float64 [3][n] or NULL:  (d2I/dx2) u for u float64 [3][n] (matrix free)
 * xt may be NULL (no inertia term in energy / grad; Hu still includes M u).
 * Errors: GIPC_ERR_INVALID_ARG, GIPC_ERR_OOM, GIPC_ERR_CUDA. */
gipc_status gipc_potential_derivs(gipc_ctx* ctx, const gipc_scene* sc_h, const double* x, const double* xt,
                                  const int32_t* stencils, const double* eps_x, int64_t k,
                                  const gipc_barrier_params* bp_h, const gipc_elastic_params* ep_h,
                                  const double* u, double* energy_h, double* grad, double* Hu, void* stream);

/* The exact Hessian M + sum_e P_e^T (d2 E_e / dx_e^2) P_e of the same potential assembled into
 * `bsr_h` (float64; capacity protocol of gipc_assemble_bsr).  It may be indefinite.
 * Synchronises once (pattern size).  Errors as gipc_assemble_bsr. */
gipc_status gipc_potential_hessian(gipc_ctx* ctx, const gipc_scene* sc_h, const double* x, const int32_t* stencils,
                                   const double* eps_x, int64_t k, const gipc_barrier_params* bp_h,
                                   const gipc_elastic_params* ep_h, gipc_bsr* bsr_h, void* stream);

/* Adjoint of one converged implicit step (x_old, v_old) -> (x_new, v_new = (x_new - x_old)/dt),
 * by implicit differentiation of grad I(x_new) = 0: with a = adj_x_new + adj_v_new / dt on free
 * vertices, solve H lambda = a (H the exact Hessian at x_new with the contacts at x_new, fixed
 * vertices filtered; modified PCG stopped as gipc_pcg does, once r.P^-1 r < prm_h->pcg_tol times
 * its start -- a ratio of squared norms, so 1e-20 asks for a 1e-10 smaller residual -- or after
 * prm_h->max_pcg iterations; at a converged step H is the Hessian at a minimiser, so it is positive
 * semidefinite on the free coordinates and PCG applies), then
 *   adj_v_old = dt M lambda                      (0 on fixed vertices)
 *   adj_x_old = M lambda - adj_v_new / dt         (adj_x_new - H lambda on fixed vertices)
 *   *adj_logE_h += -lambda . dI_elastic/dx        (= E dL/dE: Psi is linear in E at fixed nu)
 * adj_x_new / adj_v_new may be NULL (zero); adj_x_old / adj_v_old may be NULL (not written).
 * x_new must be a converged step of gipc_newton_step with the same parameters.  Synchronises.
 * Errors: GIPC_ERR_INVALID_ARG, GIPC_ERR_NOT_CONVERGED (the adjoint solve), GIPC_ERR_INDEFINITE
 * (the exact Hessian at x_new is not positive definite: x_new is not a converged minimiser; refine
 * it with gipc_newton_polish), GIPC_ERR_OOM,
 * GIPC_ERR_CUDA. */
gipc_status gipc_adjoint_step(gipc_ctx* ctx, const gipc_scene* sc_h, const double* x_new, const double* x_old,
                              const double* v_old, const gipc_step_params* prm_h, const double* adj_x_new,
                              const double* adj_v_new, double* adj_x_old, double* adj_v_old, double* adj_logE_h,
                              int* pcg_iters_h, void* stream);

/* Refinement of a step of gipc_newton_step for differentiation: Newton iterations on the same
 * incremental potential (inertia target xt = x_old + dt v_old + dt^2 g, x_old on fixed vertices)
 * with the exact Hessian instead of the projected one.  At a minimiser that Hessian is positive
 * semidefinite and Newton converges quadratically, so a step the projected method (linear
 * convergence, an energy line search that cannot resolve decreases below the rounding of I)
 * leaves at eps_d ~ 1e-6 reaches eps_polish ~ 1e-13 in a few iterations.  Each iteration:
 * contacts at x, exact gradient and Hessian (modified PCG to prm_h->pcg_tol, at most
 * prm_h->max_pcg iterations), the CCD step along d capped at 1 (slackness 0.1), x += alpha d.
 *   x      float64 [3][n], in / out;  v  float64 [3][n] or NULL: out, (x - x_old) / dt
 *   eps_polish  stop once alpha = 1 and max|d| / (l dt) <= eps_polish
 *   max_iters   at most this many iterations;  iters_h, step_h (host, may be NULL): iterations
 *               run and the last max|d| / (l dt)
 * A direction that does not descend (the exact Hessian not positive definite there) ends the
 * refinement without moving x.  Synchronises every iteration.
 * Errors: GIPC_ERR_INVALID_ARG, GIPC_ERR_NOT_CONVERGED (eps_polish not reached; x and v hold the
 * last iterate), GIPC_ERR_CAPACITY, GIPC_ERR_OOM, GIPC_ERR_CUDA. */
gipc_status gipc_newton_polish(gipc_ctx* ctx, const gipc_scene* sc_h, double* x, double* v, const double* x_old,
                               const double* v_old, const gipc_step_params* prm_h, double eps_polish, int max_iters,
                               int* iters_h, double* step_h, void* stream);

/* ------------------------------------------------------------------ profiling */

/* Kernels that a context can time with CUDA events on the stream they are
 * launched on (per-phase tracing; the events add no synchronisation). */
typedef enum {
    GIPC_PROF_PCG_SPMV = 0,      /* q = S(H c) and its partial dot products       */
    GIPC_PROF_PCG_UPDATE = 1,    /* x, r update, preconditioner, r.s              */
    GIPC_PROF_PCG_DIRECTION = 2, /* c = S(s + beta c)                             */
    GIPC_PROF_ASM_PATTERN = 3,   /* assembly: count .. rowptr (one span per call) */
    GIPC_PROF_ASM_VALUES = 4,    /* assembly: emit + value / gradient sums        */
    GIPC_PROF_CONTACTS = 5,      /* contact detection (broad phase + classify)    */
    GIPC_PROF_CCD = 6,           /* CCD step filter                               */
    GIPC_PROF_ELEMENTS = 7,      /* time step: element gradients + Hessians       */
    GIPC_PROF_ENERGY = 8,        /* time step: energies and their reductions      */
    GIPC_PROF_PCG_LOOP = 9,      /* persistent solver: all iterations of a solve  */
    GIPC_PROF_KINDS = 10
} gipc_prof_kind;

typedef struct {
    int64_t launches;   /* timed launches (spans) since gipc_profile_begin */
    double total_ms;    /* summed device time of those spans               */
} gipc_kernel_time;

/* Start (or restart) recording per-kernel spans on this context's calls. */
gipc_status gipc_profile_begin(gipc_ctx* ctx);
/* Synchronise on the recorded events and report the spans of one kind;
 * recording continues until gipc_profile_stop. */
gipc_status gipc_profile_read(gipc_ctx* ctx, int kind, gipc_kernel_time* out_h);
gipc_status gipc_profile_stop(gipc_ctx* ctx);
/* Record only one launch in `every` of `kind` (0 or 1: every launch; kept across
 * gipc_profile_begin).  Each recorded span is an event pair on the launching stream around the
 * launch, and the pair delays the next launch by a few microseconds, so the per-iteration solver
 * kernels are best sampled.  `launches` of gipc_profile_read then counts the recorded spans.
 * Errors: GIPC_ERR_INVALID_ARG. */
gipc_status gipc_profile_sampling(gipc_ctx* ctx, int kind, int every);

/* Phases of the persistent solver (tracing of gipc_pcg's single-system solve, which runs every
 * iteration in one launch).  With tracing on, every persistent solve of this context records, for
 * each of its first GIPC_TRACE_MAX_ITERS iterations, the earliest and the latest globaltimer stamp
 * over its CTAs at each phase boundary.  gipc_profile_solver_phases synchronises the device, reads
 * the stamps of the context's last traced solve and returns, per phase, the median over its
 * iterations (the first two and the last left out; at least four iterations are needed) of the
 * phase's length in microseconds, in the order of gipc_solver_phase, and the number of iterations
 * used.  A phase runs from the first CTA's start (the last CTA's for the barriers) to the last
 * CTA's end (the first CTA's exit for the barriers).  The stamps add a few global atomics per CTA
 * and phase: leave tracing off when timing.  The x update runs between a CTA's arrival at barrier
 * B and its wait, so it counts to BARRIER_B.  Errors: GIPC_ERR_INVALID_ARG (null context or output;
 * no traced solve of four or more iterations), GIPC_ERR_CUDA. */
typedef enum {
    GIPC_PHASE_PRODUCT = 0,      /* q = S(H c) and the CTA's part of c . q              */
    GIPC_PHASE_BARRIER_A = 1,    /* grid barrier after the product                      */
    GIPC_PHASE_TOTAL_A = 2,      /* c . q summed from the parts, alpha formed           */
    GIPC_PHASE_VECTOR = 3,       /* r update, s = P^-1 r and the CTA's part of r . s    */
    GIPC_PHASE_BARRIER_B = 4,    /* grid barrier after the vector phase                 */
    GIPC_PHASE_TOTAL_B = 5,      /* r . s summed, beta and the stopping test formed     */
    GIPC_PHASE_DIRECTION = 6,    /* c = S(s + beta c)                                   */
    GIPC_PHASE_BARRIER_C = 7,    /* grid barrier after the direction                    */
    GIPC_PHASE_ITERATION = 8,    /* one whole iteration                                 */
    GIPC_PHASE_COUNT = 9
} gipc_solver_phase;
#define GIPC_TRACE_MAX_ITERS 1024
gipc_status gipc_profile_solver_trace(gipc_ctx* ctx, int enable);
gipc_status gipc_profile_solver_phases(gipc_ctx* ctx, double* phase_us_h, int* iters_h);

/* Batched solves (gipc_pcg over several scenes, and so gipc_newton_step_batch) run every
 * iteration in one cooperative launch by default: the rows are spread over the CTAs by vertex,
 * a scene cut by the CTAs' ranges gets its dots summed over them in a fixed order, and four
 * bounded grid barriers separate the product, the dot parts, the update and the direction.
 * Where the grid cannot hold the batch (more than 3 x 512 vertices per CTA slot) or a CTA would
 * cut more than 64 scenes, and when gipc_pcg_batch_persistent(ctx, 0) turns it off, they run a
 * product and a per-scene update kernel per iteration instead (the product's staging variant then
 * tuned as described below).  The two differ in the summation order of the dots only.  Errors:
 * GIPC_ERR_INVALID_ARG (null context). */
gipc_status gipc_pcg_batch_persistent(gipc_ctx* ctx, int enable);

/* Run-time tuning of the batched solver's product (gipc_pcg over several scenes, and so
 * gipc_newton_step_batch).  The product q = S(H c) streams the matrix in SELL-32 slices; how
 * many block columns a warp stages per copy (U), how many warps share a CTA (W) and how many
 * copies are in flight (NS) trade shared memory, occupancy and latency differently on different
 * batches.  While tuning is on (the default), a context runs its first batched solves of each
 * precision and size class floor(log2(nnzb)) with each of GIPC_SPMV_VARIANTS staging variants in
 * turn, a whole chunk of iterations at a time (product and scene update, so the overlap of
 * consecutive launches counts), timed by CUDA events on the stream; chunks after which the solve
 * has ended are not counted.  Once every variant has GIPC_SPMV_TUNE_SAMPLES timed iterations the
 * fastest per iteration is kept for that class.  The product of every row is formed in the same order whatever the variant, and
 * the batched solver sums its dot products per scene itself, so results do not depend on the
 * choice.  gipc_spmv_autotune(ctx, 0) fixes variant 0.  gipc_spmv_tunings copies up to `cap`
 * classes the context has measured (precision, size class, chosen variant or -1 while measuring,
 * each variant's U, W, NS, timed iterations and mean microseconds per iteration) to out_h and
 * their count to count_h.
 * Errors: GIPC_ERR_INVALID_ARG (null context; null out_h with cap > 0; null count_h). */
#define GIPC_SPMV_VARIANTS 4
#define GIPC_SPMV_TUNE_SAMPLES 32
typedef struct {
    int precision;                      /* GIPC_FP64 or GIPC_MIXED          */
    int size_class;                     /* floor(log2(nnzb)) of the systems */
    int chosen;                         /* variant in use; -1 while timing  */
    int U[GIPC_SPMV_VARIANTS];          /* block columns per staged copy    */
    int W[GIPC_SPMV_VARIANTS];          /* warps per CTA                    */
    int NS[GIPC_SPMV_VARIANTS];         /* copies in flight per warp        */
    int samples[GIPC_SPMV_VARIANTS];    /* timed iterations                 */
    double mean_us[GIPC_SPMV_VARIANTS]; /* per iteration                    */
} gipc_spmv_tuning;
gipc_status gipc_spmv_autotune(gipc_ctx* ctx, int enable);
gipc_status gipc_spmv_tunings(gipc_ctx* ctx, gipc_spmv_tuning* out_h, int cap, int* count_h);

#ifdef __cplusplus
}
#endif
#endif /* GIPC_H */

/*
 * os3d — invertible orientation scores of 3D images on one GB300 (sm_103a).
 *
 * C ABI of the transform of Janssen, Duits and Breeuwer, "Invertible
 * Orientation Scores of 3D Images" (arXiv 1505.07690):
 *   cake wavelets  psi_hat_i(w) = G(|w|) h(w_hat . n_i),  h = sum_l c_l P_l
 *                  (Sec. 3.1 radial window and B-spline orientation
 *                  distribution, Sec. 3.2 zonal SH fit, Funk transform,
 *                  anti-symmetrisation and steering, Eq. Rotationh);
 *   forward        U_i = IDFT[ f_hat conj(psi_hat_i) ]      (Eq. construction1Discrete);
 *   exact inverse  f = Re IDFT[ max(M,eps)^-1 sum_i psi_hat_i DFT(U_i) ],
 *                  M = sum_i |psi_hat_i|^2                   (Eq. Reconstruction1Discrete,
 *                                                             clamp of Sec. 3.1);
 *   adjoint        W^* G = Re IDFT[ sum_i psi_hat_i DFT(G_i) ] (Sec. 4.1, App. A).
 *
 * Discrete conventions: the DFT is unnormalised with kernel exp(-i w.x) (the
 * paper's sign); w_j = 2 pi k_j / n_j on the signed DFT index, so the Nyquist
 * frequency is rho_N = pi; psi_hat vanishes outside the ball |w| < pi (the
 * ball-limited images of Sec. 2 with varrho = rho_N); at w = 0 the angular
 * factor is the spherical mean c_0 of h. The continuous constants (2 pi)^(3/2)
 * and d sigma = 4 pi / N_o cancel in the exact inverse and are absorbed into
 * the normalisation kappa of c, chosen so that the spherical mean of
 * sum_i h(w_hat . n_i)^2 is 1 (the paper's aim M ~ 1, Sec. 2).
 *
 * Layout: volumes are row-major (nz, ny, nx), x fastest. A score U holds
 * batch x N_o volumes, index ((b * N_o + i) * nz + z) * ny * nx + y * nx + x,
 * each element complex: OS3D_U_C64 = interleaved float (re, im) (8 bytes),
 * OS3D_U_BF16X2 = interleaved bfloat16 (re, im), round to nearest even
 * (4 bytes). Re U = line response, Im U = edge response (Sec. 3, requirement 6).
 *
 * Ownership: the caller owns every data buffer (device pointers). A bank owns
 * its coefficients and per-voxel factors until os3d_destroy_bank, and also a
 * default workspace, which the first transform call made with a NULL
 * workspace allocates (cudaMalloc, so that call must not be under stream
 * capture; ENOMEM if it fails). Callers that always pass a workspace never
 * cause that allocation.
 * Ordering: every call that takes a stream only enqueues work on it and
 * returns; none synchronises the device, except os3d_make_wavelets, which
 * synchronises its own stream once (it copies the fitted coefficients back).
 * Errors: every entry point returns an os3d_status; arguments are checked
 * before any launch; nothing aborts or throws across the ABI.
 * Alignment: the device buffers of the transform calls (images, scores,
 * gradients) must start on 16-byte boundaries (EINVAL otherwise); the kernels
 * move two adjacent complex values per access.
 * Devices: a bank belongs to the device that was current at its creation;
 * calls on it must be made with that device current.
 * Concurrency: calls that share a workspace (including the bank's default
 * one, used when the workspace argument is NULL) must be ordered on one
 * stream; give concurrent calls distinct workspaces of os3d_bank_info's
 * workspace_bytes.
 */
#ifndef OS3D_H
#define OS3D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  OS3D_OK = 0,
  OS3D_EINVAL = 1,       /* a NULL pointer, a size or a parameter out of range   */
  OS3D_ENOMEM = 2,       /* device allocation failed                             */
  OS3D_ECUDA = 3,        /* a CUDA call failed (launch or copy)                  */
  OS3D_ETIMEOUT = 4,     /* reserved for bounded waits of the serving loop       */
  OS3D_EUNSUPPORTED = 5  /* grid size without a compiled FFT plan                */
} os3d_status;

typedef enum { OS3D_U_C64 = 0, OS3D_U_BF16X2 = 1 } os3d_udtype;

/* Wavelet parameters (Sec. 3.1 and 3.2; defaults from os3d_default_params). */
typedef struct {
  int k;            /* order of the B-spline orientation distribution A = B^k(theta/s_theta); 0..8 */
  double s_theta;   /* angular width s_theta > 0                                     */
  int L;            /* maximal Legendre / SH degree, 0..32                            */
  int N;            /* order of the radial window g = M_N, 0..64                      */
  double gamma;     /* inflection point of g at gamma * rho_N, 0 < gamma < 1          */
  double eps;       /* clamp M -> max(M, eps) of the inverse, eps > 0                */
  int fit_mode;     /* 1: least squares on the order-15 icosahedral tessellation
                       (the paper's pseudo-inverse); 0: L2 projection (Gauss-Legendre) */
  int block_slots;  /* orientation pairs per launch block, 0 = automatic (11), else 1..12 */
  int overlap;      /* 1: consecutive blocks alternate between two internal streams of the
                       bank (forked from and joined to the caller's stream); 0: every launch
                       on the caller's stream (for callers running many transforms at once) */
  int profile;      /* angular part h: 0 = cake wavelet, h = F A + antisym(A) (line and edge
                       detector, Sec. 3.1, Eq. CakeWaveletRe / Eq. Antisymmetrize);
                       1 = h = A itself (plate and edge detector, Sec. 3.1, Fig. 3)   */
} os3d_params;

typedef struct os3d_bank os3d_bank; /* opaque, library-owned */

/* Defaults: k = 2, s_theta = 0.7, L = 16, N = 8, gamma = 0.8, eps = 1e-4,
 * fit_mode = 1, block_slots = 0, overlap = 1, profile = 0. Host only. */
os3d_status os3d_default_params(os3d_params* p);

/* Orientation set of Sec. 2.1: an icosahedron (vertices: cyclic permutations
 * of (0, +-1, +-phi), normalised) subdivided `subdiv` times by edge midpoints
 * projected onto S^2: 12, 42, 162, 642 ... unit vectors; both members of every
 * antipodal pair are kept. Order: the representatives (z > 0, or z = 0 and
 * y > 0, or z = y = 0 and x > 0) by decreasing z, then increasing azimuth
 * atan2(y, x) in (-pi, pi]; then their antipodes in the same order, so that
 * n_{i + N_o/2} = -n_i. `out` (host) receives n_o x 3 doubles (x, y, z);
 * `capacity` is its length in vectors. Host only; subdiv 0..4.
 * Returns OS3D_EINVAL if subdiv is out of range or capacity is too small
 * (then *n_o still receives the required count). */
os3d_status os3d_icosa_orientations(int subdiv, double* out, int capacity, int* n_o);

/* The other platonic-solid sampling of Sec. 2.1: an octahedron (vertices
 * +-e_x, +-e_y, +-e_z) subdivided `subdiv` times in the same way: 6, 18, 66,
 * 258, 1026, 4098 unit vectors, in the same canonical order. It is mapped onto
 * itself by the 90-degree rotations about the coordinate axes, which on a
 * cubic grid permute the channels of a score exactly. Host only; subdiv 0..5;
 * errors as os3d_icosa_orientations. */
os3d_status os3d_octa_orientations(int subdiv, double* out, int capacity, int* n_o);

/* Builds the wavelet bank for a grid dims = {nz, ny, nx} and the orientation
 * set `orient` (host, n_o x 3 doubles, unit vectors, x y z). Steps (all on
 * the device current at the call, stream-ordered on `stream`):
 *  (a1) zonal fit b_l of A (FP64 kernel), Funk transform c^e_l = 2 pi P_l(0) b_l,
 *       anti-symmetrisation c^o_l = (1 - (-1)^l) b_l, c = kappa (c^e + c^o)
 *       (Sec. 3.2); with profile = 1, c = kappa b;
 *  (a3) M = G^2 sum_i h(w_hat . n_i)^2 in FP64 and the factors
 *       G / n^3 and G / (n^3 max(M, eps)) stored as float (Sec. 2.1, 3.1).
 * Antipodal pairs in `orient` are detected (|n_i + n_j| < 1e-9) and share
 * one transform in the forward and inverse passes.
 * Supported axis lengths: 16, 32, 48, 64, 96, 128, 160 and 256 on every axis.
 * Square (ny, nx) planes of side <= 128, 128 x 160 planes and 256^2 planes
 * use the fused 2D plane pass (a whole plane per CTA, or for 256^2 an eighth
 * of a plane per CTA on clusters of 8); other planes use separate x and y
 * pencil passes.
 * Errors: EINVAL (NULL, n_o < 1, a non-unit orientation, parameter out of
 * range), EUNSUPPORTED (grid), ENOMEM, ECUDA. `stream` may be NULL (legacy
 * default stream). */
os3d_status os3d_make_wavelets(const int dims[3], const double* orient, int n_o,
                               const os3d_params* p, void* stream, os3d_bank** out);

/* Forward transform (a4, a5): U = W f for `batch` real volumes f (device,
 * batch x nz x ny x nx float) into U (device, batch x N_o x nz x ny x nx,
 * udtype). Valid for real f: an antipodal pair is written as U_b = conj(U_a).
 * `workspace` (device, os3d_bank_info's workspace_bytes, 256-byte aligned)
 * or NULL for the bank's own. f must be 16-byte aligned. Errors: EINVAL, ECUDA. */
os3d_status os3d_forward(const os3d_bank* bank, const float* f, int batch, void* U,
                         os3d_udtype udtype, void* workspace, void* stream);

/* Exact inverse (a6): f_out = Re IDFT[ max(M,eps)^-1 sum_i psi_hat_i DFT(U_i) ]
 * for `batch` scores U (device, layout as above) into f_out (device, float).
 * Any U is accepted (not only ranges of W). Errors: EINVAL, ECUDA. */
os3d_status os3d_inverse(const os3d_bank* bank, const void* U, os3d_udtype udtype, int batch,
                         float* f_out, void* workspace, void* stream);

/* Adjoint (a7): grad_f = Re IDFT[ sum_i psi_hat_i DFT(G_i) ] = Re W^* G for
 * `batch` score-shaped G (device). For a real loss L(U) with G = dL/dconj(U)
 * in PyTorch's convention this is dL/df. Errors: EINVAL, ECUDA. */
os3d_status os3d_adjoint(const os3d_bank* bank, const void* G, os3d_udtype udtype, int batch,
                         float* grad_f, void* workspace, void* stream);

/* Weighted adjoint (the adjoint of Sec. 4.1 and App. A applied to the
 * gradient of the weighted energy): grad_f = Re W^*(2 g w U), the gradient
 * with respect to a real image f of g sum w |U|^2 at U = W f (see
 * os3d_weighted_energy), i.e.
 * os3d_adjoint of os3d_weighted_energy_grad's G without G being stored: the
 * plane pass multiplies each element of U by 2 g w as it loads it. U (device,
 * batch complex64 scores), w (device float, one weight per complex element,
 * U's layout, 16-byte aligned), g (device float scalar). Errors: EINVAL,
 * EUNSUPPORTED (BF16 U, or a plane the plane pass does not hold: there
 * os3d_weighted_energy_grad and os3d_adjoint give the same result), ECUDA. */
os3d_status os3d_adjoint_weighted(const os3d_bank* bank, const void* U, const float* w,
                                  const float* g, os3d_udtype udtype, int batch, float* grad_f,
                                  void* workspace, void* stream);

/* Weighted energy of the score of an image and its gradient in one sweep,
 * without storing the score: L = sum w |W f|^2 (the weighted squared
 * L_2(R^3 x S^2) norm of Sec. 2) and grad_f = Re W^*(2 g w W f), its gradient
 * with respect to the real image f scaled by g, for `batch` volumes f
 * (device float, batch x nz x ny x nx). Per block of orientation pairs the
 * forward z-pass, one plane pass that forms U_a = W f in shared memory, sums
 * (w_a + w_b) |U_a|^2 and replaces U_a by 2 g (w_a + w_b) U_a (U_b = conj U_a,
 * w real), and the adjoint's z-pass (the structure of os3d_upsilon with the
 * soft threshold replaced by the weighting). w (device float, the score's
 * layout: batch x N_o x nz x ny x nx, 16-byte aligned); g (device float) or
 * NULL for 1. `scratch` (device, at least os3d_score_energy_scratch doubles,
 * 8-byte aligned, not shared with a concurrent call): scratch[0] receives L in
 * double precision (one FP64 sum per plane and orientation pair, added in
 * index order: bit-identical from call to call), `loss` (device float or NULL)
 * L rounded to float. Planes of the plane pass (square 16^2 to 128^2, 256^2,
 * 128 x 160; those of os3d_upsilon's fused plane pass); elsewhere EUNSUPPORTED
 * (os3d_forward, os3d_weighted_energy and os3d_adjoint_weighted or
 * os3d_adjoint give the same results). Errors: EINVAL, EUNSUPPORTED, ECUDA. */
os3d_status os3d_score_energy_grad(const os3d_bank* bank, const float* f, const float* w,
                                   const float* g, int batch, float* loss, float* grad_f,
                                   double* scratch, size_t scratch_doubles, void* workspace,
                                   void* stream);

/* Doubles of scratch os3d_score_energy_grad needs for `batch` volumes:
 * 1 + batch x (orientation pairs and unpaired orientations) x nz x (CTAs per
 * plane: 8 for 256^2 planes, else 1). */
os3d_status os3d_score_energy_scratch(const os3d_bank* bank, int batch, size_t* doubles);

/* y = g x over `count` floats (device, 16-byte aligned; y may be x), g read
 * on the device: the chain-rule factor of an upstream gradient. Errors:
 * EINVAL, ECUDA. */
os3d_status os3d_scale_by(const float* x, float* y, long long count, const float* g,
                          void* stream);

/* Approximate reconstruction (Eq. Reconstruction2Approximation):
 * f_out = w Re sum_i U_i with the discrete measure w = 1 / (N_o c_0), the
 * value that makes the orientation sum of the wavelets exactly 1 at w = 0
 * (where every psi_hat_i equals c_0), i.e. the paper's condition
 * (2 pi)^(3/2) int F[psi_n] d sigma ~ 1 read at the origin. No Fourier
 * transform: one streaming pass over U (device, batch scores) into f_out
 * (device, batch x nz x ny x nx float, 16-byte aligned). Errors: EINVAL
 * (also when c_0 = 0), ECUDA. */
os3d_status os3d_approx_reconstruct(const os3d_bank* bank, const void* U, os3d_udtype udtype,
                                    int batch, float* f_out, void* stream);

/* Projection onto the space of orientation scores (App. A, corollary):
 * P_psi U = W W^{*,ext} U, with W^{*,ext} the exact reconstruction (the
 * adjoint extended to the embedding space with the M_psi inner product), i.e.
 * os3d_inverse followed by os3d_forward, per volume. U and U_out (device,
 * batch scores of udtype) may be the same buffer. The intermediate image is
 * kept in the workspace. Errors: EINVAL, ECUDA. */
os3d_status os3d_project(const os3d_bank* bank, const void* U, os3d_udtype udtype, int batch,
                         void* U_out, void* workspace, void* stream);

/* Soft thresholding Phi(U) = |U|^p sgn(U) of Sec. 4.1 (Fig. 6 uses p = 1.5),
 * applied to the real (line) and imaginary (edge) parts separately, on
 * `count` complex elements (a multiple of 4) of `in` into `out` (device,
 * 16-byte aligned, may be equal). BF16 results round to nearest even.
 * Errors: EINVAL (count, alignment, p <= 0 or not finite), ECUDA. */
os3d_status os3d_soft_threshold(const void* in, void* out, os3d_udtype udtype, long long count,
                                double power, void* stream);

/* Weighted energy of a score, L = sum_e w_e |U_e|^2 over `count` complex
 * elements (a multiple of 4): the squared L_2(R^3 x S^2) norm of the score in
 * the norm-preservation identity of Sec. 2 (M_psi = 1 gives ||f||^2 =
 * ||W f||^2), with real weights w (device float, one per complex element,
 * same layout as U) or w = NULL for w = 1; the loss whose gradient feeds
 * os3d_adjoint when the transform is differentiated. U, w 16-byte aligned.
 * `scratch` (device, OS3D_ENERGY_SCRATCH_DOUBLES doubles, 8-byte aligned, not
 * shared with a concurrent call): scratch[0] receives L in double precision;
 * if `loss` (device float) is not NULL it receives L rounded to float. Terms
 * are summed in FP32 over 16 elements and in FP64 above, on a grid fixed by the
 * device's SM count, with no atomics: the result is bit-identical from call to
 * call on one device. count = 0 writes L = 0 (U and w may then be NULL).
 * Errors: EINVAL (count, alignment, NULL scratch, NULL U with count > 0),
 * ECUDA. */
#define OS3D_ENERGY_SCRATCH_DOUBLES 4097
os3d_status os3d_weighted_energy(const void* U, const float* w, os3d_udtype udtype,
                                 long long count, double* scratch, float* loss, void* stream);

/* Gradient of the weighted energy in PyTorch's convention for complex inputs
 * (dL/dconj(U) x 2): G = 2 g w U, with the upstream scalar g read from the
 * device (float, e.g. the incoming gradient of the loss) and w as above (NULL
 * for 1). G (device, udtype of U, 16-byte aligned) may be U. BF16 results round
 * to nearest even. count = 0 does nothing. Errors: EINVAL (count, alignment,
 * NULL pointers with count > 0), ECUDA. */
os3d_status os3d_weighted_energy_grad(const void* U, const float* w, os3d_udtype udtype,
                                      long long count, const float* g, void* G, void* stream);

/* Score-domain processing with soft thresholding (Sec. 4.1):
 * Upsilon f = W^{*,ext} Phi W f = W^* P_psi Phi W f, the exact (clamped)
 * reconstruction of the soft-thresholded score, for `batch` real volumes f
 * into f_out (device, float). Equal to os3d_forward, os3d_soft_threshold and
 * os3d_inverse in sequence (complex64 scores), but the score is never
 * stored: per block of orientation pairs the thresholding runs between the
 * inverse and the forward 2D DFT of each plane in one kernel, so the call
 * needs only the bank's workspace. Errors: EINVAL, ECUDA. */
os3d_status os3d_upsilon(const os3d_bank* bank, const float* f, int batch, float* f_out,
                         double power, void* workspace, void* stream);

/* Linear left-invariant diffusion on R^3 x| S^2 (Sec. 4.1 with a constant
 * diagonal D_ij): dW/dt = [D11 (A1^2 + A2^2) + D33 A3^2 + D44 (A4^2 + A5^2)] W,
 * where for a function of (x, n) A3 = n . grad_x, A1^2 + A2^2 =
 * Laplace_x - (n . grad_x)^2 and A4^2 + A5^2 is the Laplace-Beltrami
 * operator of S^2 in n (D66 drops out by the equivalence relation). */
typedef struct {
  double t;         /* diffusion time >= 0 (Fig. 5: t = 10)                          */
  int steps;        /* Strang splitting steps K, 1..4096                             */
  double D11;       /* spatial diffusion perpendicular to n, >= 0                    */
  double D33;       /* spatial diffusion along n, >= 0                               */
  double D44;       /* angular diffusion, >= 0                                       */
  int sh_degree;    /* degree of the discrete Laplace-Beltrami operator, 0..15; 0 = the
                       largest l with (l+1)^2 <= N_o whose real spherical harmonics are
                       linearly independent on the orientation set                  */
} os3d_diffusion;

/* t = 10, steps = 8, D11 = 0, D33 = 1, D44 = 0.01, sh_degree = 0. Host only. */
os3d_status os3d_default_diffusion(os3d_diffusion* d);

/* The angular propagator exp(tau L) of the discrete Laplace-Beltrami operator
 * on n orientations `orient` (host, n x 3) into E (host, n x n doubles,
 * row-major), in FP64: E = I + Y (exp(tau Lambda) - I) (Y^T Y)^-1 Y^T with
 * the real spherical harmonics Y up to degree `sh_degree` (0 = automatic, as
 * in os3d_diffusion). *degree_used (may be NULL) receives the degree. Host
 * only. Errors: EINVAL (NULL, n < 1, tau < 0, dependent harmonics). */
os3d_status os3d_angular_propagator(const double* orient, int n, int sh_degree, double tau,
                                    double* E, int* degree_used);

/* Enhancement Upsilon f = W^{*,ext} Phi_t W f with the linear diffusion Phi_t
 * (Sec. 4.1), for `batch` real volumes f into f_out (device, float). The
 * evolution is integrated in the Fourier domain of x: per orientation the
 * spatial generators are the exact factor exp(-dt r_i(w)), r_i(w) = D11 (|w|^2
 * - (w.n_i)^2) + D33 (w.n_i)^2; the angular generator is the discrete
 * Laplace-Beltrami operator L = Y diag(-l(l+1)) Y^+ of the real spherical
 * harmonics Y on the orientation set, applied as exp(dt D44 L) (FP64 on the
 * host); K Strang steps of dt = t/K (half spatial, angular, half spatial).
 * Because every operator in the cascade commutes with translations, the
 * whole of W^{*,ext} Phi_t W acts on f_hat through one real factor per
 * frequency: the score is never formed and no per-orientation transform
 * runs. Sets of at most 68 orientations run the product E v on the CUDA cores
 * (one GPU thread per frequency and row block); larger sets, up to 176
 * orientations (the 162 set), on the tensor cores (tcgen05, half-precision
 * operands split into high and low parts, FP32 accumulation; 128 frequencies
 * per step of one CTA), with bounded waits counted by os3d_bank_wait_errors.
 * Errors: EINVAL (NULL, parameters out of range, dependent harmonics at the
 * requested degree), EUNSUPPORTED (more than 176 orientations, or a workspace
 * too small for the propagator), ECUDA. */
os3d_status os3d_enhance_linear(const os3d_bank* bank, const float* f, int batch, float* f_out,
                                const os3d_diffusion* d, void* workspace, void* stream);

/* Sizes: workspace bytes one call needs, and the device bytes one volume
 * occupies through forward + inverse: its complex64 score (N_o x nz x ny x nx
 * x 8) plus the input and the output image (2 x nz x ny x nx x 4); a BF16X2
 * score takes half of the score's part. Either pointer may be NULL. Host only. */
os3d_status os3d_bank_info(const os3d_bank* bank, size_t* workspace_bytes,
                           size_t* footprint_bytes_per_volume);

/* Device bytes the bank itself holds now: its three per-voxel float tables,
 * the in-ball frequency list and, once allocated, its default workspace.
 * Host only. Errors: EINVAL (NULL). */
os3d_status os3d_bank_resident_bytes(const os3d_bank* bank, size_t* bytes);

/* Bounded waits: the kernels that wait on an mbarrier (the tensor-core
 * diffusion) give up after 1 s of global time, count the event in a device
 * counter of the bank and carry on (their results are then invalid).
 * *count receives the counter (synchronous copy); reset != 0 sets it back to
 * 0. Errors: EINVAL (NULL, another device current), ECUDA. */
os3d_status os3d_bank_wait_errors(const os3d_bank* bank, unsigned* count, int reset);

/* Copies of bank data for inspection: the Legendre coefficients b (of A) and
 * c (of h = h_Re + h_Im, normalised), L + 1 doubles each (host); and, on the
 * device, M^-1 = 1/max(M, eps) inside the ball (0 outside) as nz*ny*nx
 * floats, stream-ordered. Either output pointer may be NULL. */
os3d_status os3d_bank_coefficients(const os3d_bank* bank, double* b, double* c);
os3d_status os3d_bank_minv(const os3d_bank* bank, float* minv, void* stream);

os3d_status os3d_destroy_bank(os3d_bank* bank);
const char* os3d_status_string(os3d_status s);

/* ---- serving (no counterpart in the paper) --------------------------------
 * A server owns a device arena of arena_bytes, allocated once at creation, and
 * a worker thread. Each request is one host volume f (nz*ny*nx floats) with
 * the icosahedral orientation set of `subdiv` subdivisions: the server copies
 * f to the device, runs os3d_forward into a score held in the arena, then
 * os3d_inverse, and copies the reconstruction to f_out (host). Requests are
 * admitted in arrival order as soon as one of max_inflight stream slots and
 * the request's footprint (score + two images + workspace) in the arena are
 * free; admitted requests run concurrently. Wavelet banks are made on first
 * use per (grid, orientation set) with the server's parameters and cached;
 * when the banks' resident bytes (os3d_bank_resident_bytes) would exceed
 * bank_cache_bytes, idle banks (no request in flight) are destroyed, least
 * recently used first. Placement: each bank remembers up to 2 x max_inflight
 * arena offsets ("homes") where its requests ran; a request takes the first
 * free home of its bank, else the first free range that fits (recorded as a
 * new home while there is room). f and f_out must stay valid until the request is
 * complete and should be page-locked (pageable host memory makes the copies,
 * and with them the worker thread, synchronous). The server must be created,
 * used and destroyed with one device current. */
typedef struct {
  size_t arena_bytes;  /* device memory for in-flight requests                  */
  int max_inflight;    /* concurrent requests (streams), 1..64                  */
  int udtype;          /* score storage of every request: OS3D_U_C64 or BF16X2  */
  int use_graphs;      /* 1: the kernels of forward + inverse for one (bank, home)
                          are captured as a CUDA graph on the first request placed
                          there and replayed by every later one (up to 512 graphs,
                          then the cache is cleared; a bank's graphs go with it);
                          requests placed outside their bank's homes run with
                          direct launches. 0: direct launches only                */
  size_t bank_cache_bytes; /* budget for the resident bytes of cached banks, > 0   */
} os3d_server_config;
typedef struct os3d_server os3d_server;

/* arena_bytes = 16 GiB, max_inflight = 4, udtype = OS3D_U_C64, use_graphs = 1,
 * bank_cache_bytes = 4 GiB. Host only. */
os3d_status os3d_server_default_config(os3d_server_config* cfg);
/* Errors: EINVAL (config out of range), ENOMEM (arena), ECUDA. p may be NULL
 * (defaults). */
os3d_status os3d_server_create(const os3d_server_config* cfg, const os3d_params* p,
                               os3d_server** out);
/* Queues a request and returns its ticket at once. EINVAL for bad arguments;
 * a grid without a plan or a request larger than the arena completes with
 * that status (EUNSUPPORTED, ENOMEM) instead. */
os3d_status os3d_server_submit(os3d_server* s, const int dims[3], int subdiv, const float* f,
                               float* f_out, long long* ticket);
/* Waits at most timeout_s seconds for the request: OS3D_ETIMEOUT if it is not
 * complete by then (the ticket stays valid), else the request's status; then
 * *latency_ms (may be NULL) is the time from submission to completion and the
 * ticket is released. */
os3d_status os3d_server_wait(os3d_server* s, long long ticket, double timeout_s,
                             double* latency_ms);
/* Counters since creation: completed requests, graphs captured, graph replays
 * (requests served by an already captured graph). Any pointer may be NULL. */
os3d_status os3d_server_stats(os3d_server* s, long long* completed, long long* graphs_captured,
                              long long* graph_replays);
/* Finishes every queued and in-flight request, then frees the server. */
os3d_status os3d_server_destroy(os3d_server* s);

/* ---- forward transform without a workspace (no counterpart in the paper) --
 * os3d_forward_static computes exactly what os3d_forward computes, but keeps
 * all of its scratch in a fixed array inside the library instead of a
 * workspace, and allocates nothing: no cudaMalloc, cudaFree or allocating
 * library call. It is meant for callers that cannot allocate device memory
 * when they run the transform (device memory owned by a framework's pool
 * allocator that may not be bypassed; latency-critical loops where a
 * cudaMalloc, which can synchronise the device, is not acceptable). The bank
 * itself is still made beforehand by os3d_make_wavelets.
 * Limits: volumes of at most OS3D_STATIC_MAX_VOXELS voxels (64^3); larger
 * banks are rejected with OS3D_EINVAL. The array (3 x OS3D_STATIC_MAX_VOXELS
 * complex floats, 6 MiB) is held by every GPU that loads the library until
 * the process exits. The first call in each CUDA context of a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture. A context created
 * anew (for instance after cudaDeviceReset) is recognised by its unique id and
 * gets a fresh lookup on its first call. All calls share the one array and it
 * keeps the last call's contents (every element is overwritten before it is
 * read, so nothing needs clearing); calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * Orientation pairs are processed one at a time on `stream` (no side
 * streams). Arguments and errors otherwise as os3d_forward. */
#define OS3D_STATIC_MAX_VOXELS (64 * 64 * 64)
os3d_status os3d_forward_static(const os3d_bank* bank, const float* f, int batch, void* U,
                                os3d_udtype udtype, void* stream);


/* ---- diagnostics (no counterpart in the paper) ---------------------------
 * Kernel kinds of the transform: the xy-passes (2D DFT of one z-plane with
 * the score store or load fused) and the z-passes (DFT along z with the
 * wavelet evaluation, the orientation sum or a per-voxel factor fused). */
enum {
  OS3D_KIND_XY_FWD_REAL = 0,   /* forward: DFT_xy of the real image            */
  OS3D_KIND_XY_FWD_SCORE = 1,  /* forward: IDFT_xy and store of U_a, U_b       */
  OS3D_KIND_XY_INV_SCORE = 2,  /* inverse: load of U_a, U_b and DFT_xy         */
  OS3D_KIND_XY_INV_REAL = 3,   /* inverse: IDFT_xy and store of the real image */
  OS3D_KIND_Z_FWD_PREP = 4,    /* forward: DFT_z and the factor G / n^3        */
  OS3D_KIND_Z_FWD_SCORE = 5,   /* forward: wavelet evaluation and IDFT_z       */
  OS3D_KIND_Z_INV_SCORE = 6,   /* inverse: DFT_z, wavelet and orientation sum  */
  OS3D_KIND_Z_INV_FINAL = 7,   /* inverse: factor G / (n^3 max(M,eps)), IDFT_z */
  OS3D_KIND_XY_SOFT = 8,       /* Upsilon: IDFT_xy, soft threshold, DFT_xy     */
  OS3D_KIND_APPROX = 9,        /* approximate reconstruction: orientation sum  */
  OS3D_KIND_SOFT = 10,         /* soft threshold of a stored score             */
  OS3D_KIND_ENHANCE = 11,      /* linear diffusion: per-frequency integration  */
  OS3D_KIND_ENERGY = 12,       /* weighted energy: partial sums and final sum  */
  OS3D_KIND_ENERGY_GRAD = 13,  /* weighted energy: gradient 2 g w U            */
  OS3D_KIND_COUNT = 14
};

/* Self-test of the bounded waits (diagnostic): one CTA of 64 threads waits on
 * an mbarrier with a limit of limit_s seconds (0 < limit_s <= 10); with
 * arrive != 0 the barrier is completed first, otherwise nothing arrives and
 * every thread's wait runs out. *timeouts receives the number of threads
 * whose wait ran out (64 or 0). Synchronous; allocates and frees 4 device
 * bytes. The context stays usable afterwards. Errors: EINVAL, ENOMEM, ECUDA. */
os3d_status os3d_wait_selftest(double limit_s, int arrive, unsigned* timeouts);

/* Number of kernels this library has launched in this process. Host only. */
unsigned long long os3d_launch_count(void);

/* While enabled (on != 0), each kernel launch is bracketed by two CUDA events
 * recorded on its stream. os3d_profile_read synchronises on the recorded
 * events and returns, for one kind, the launches and total milliseconds
 * since the last os3d_profile_reset. */
os3d_status os3d_profile_enable(int on);
os3d_status os3d_profile_read(int kind, unsigned long long* launches, double* ms);
os3d_status os3d_profile_reset(void);
const char* os3d_kernel_kind_name(int kind);

#ifdef __cplusplus
}
#endif
#endif /* OS3D_H */

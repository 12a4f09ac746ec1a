/*
 * ivc.h -- C ABI of the GB300 (sm_103a) inline 3-vector compression library.
 *
 * Method: Trojak & Witherden, "Inline Vector Compression for Computational
 * Physics" (arXiv:2003.02633).  A single-precision 3-vector (12 bytes) is
 * stored in one 64-bit word: the magnitude r = |x| in a reduced float format
 * and the spherical angles theta = atan2(y, x), phi = acos(z / r) quantised to
 * integers (Sec. 2.1, Eq. cart2sphere / a_disc / a_inv; Sec. 2.3 magnitude
 * format; Fig. comp_regimes bit layouts).  The fused kernels decompress,
 * apply an FP32 elementwise operation and recompress (Sec. 5).
 *
 * Conventions shared by every entry point
 *   - Pointers marked "device" are device (or managed) memory of the current
 *     CUDA device; the caller owns every buffer.  Entry points allocate
 *     nothing per call; the first call with a given format on a device builds
 *     that format's small trigonometric tables once and keeps them until
 *     ivc_release_tables() or process exit.
 *   - Packed words are uint64_t, 8-byte aligned.  FP32 arrays are 4-byte
 *     aligned.  Wider (16-byte) vector accesses are used when pointers and
 *     sizes allow; other alignments take a scalar path.
 *   - Every call is asynchronous on `stream` (NULL = the legacy default
 *     stream) and returns a status: IVC_OK, or an error for bad arguments,
 *     a bad format, misaligned pointers or a failed launch.  No call aborts or
 *     traps.  n == 0 returns IVC_OK without launching.
 *   - Elementwise operations may run in place (c == a, y updated in place,
 *     v_out == v); partially overlapping ranges are not allowed.
 *   - Results do not depend on launch configuration.
 */
#ifndef IVC_H
#define IVC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ivc_stream_t; /* same type as cudaStream_t */

typedef enum {
  IVC_OK = 0,
  IVC_ERR_ARG = 1,        /* null pointer with n > 0, n < 0, bad enum value  */
  IVC_ERR_FORMAT = 2,     /* invalid or unsupported ivc_format              */
  IVC_ERR_ALIGN = 3,      /* pointer not aligned to its element size        */
  IVC_ERR_CUDA = 4,       /* a CUDA runtime call or launch failed           */
  IVC_ERR_TIMEOUT = 5,    /* a bounded device loop ran out of iterations    */
  IVC_ERR_NOMEM = 6,      /* workspace too small / table allocation failed  */
  IVC_ERR_UNSUPPORTED = 7 /* combination not implemented                     */
} ivc_status;

typedef enum { IVC_AOS = 0, IVC_SOA = 1 } ivc_layout;
/* AoS: xyz[3*i + k].  SoA: xyz[k*ld + i] (ld >= n, three rows). */

typedef enum {
  IVC_MAP_UNIFORM = 0,   /* Eq. (a_disc): n = nint(n_max psi)                 */
  IVC_MAP_TANH = 1,      /* Sec. 2.5: n = nint(m n_max [tanh(g(2psi-1)) + c]) */
  IVC_MAP_FRACSPLIT = 2  /* Eq. (q_split): n_p = n_phi (n_theta_max+1) + n_theta */
} ivc_map;

/* Bit layout <s,e,m>-p-t of Fig. (comp_regimes): fields from the most
 * significant bit: [sign s][exponent e][mantissa m][n_phi p][n_theta t].
 * n_theta_max = 2^t - 1, n_phi_max = 2^p - 1 (Sec. 2.4: the largest value
 * the field holds).  For IVC_MAP_FRACSPLIT the p + t low bits hold
 * n_p = n_phi (n_theta_max + 1) + n_theta with n_phi_max + 1 = nphi_max_p1
 * and n_theta_max + 1 = floor(2^(p+t) / nphi_max_p1).
 * Exponent field E: 0 = zero vector, 1 .. 2^e - 2 normal with
 * r = 2^(E - exp_bias) (1 + mantissa / 2^m), 2^e - 1 = non-finite. */
typedef struct {
  int32_t sign_bits;      /* 0 or 1 (a stored sign bit of r, always 0)        */
  int32_t exp_bits;       /* 2 .. 8                                           */
  int32_t man_bits;       /* 1 .. 23; r's FP32 mantissa is truncated to this  */
  int32_t phi_bits;       /* p                                                 */
  int32_t theta_bits;     /* t;  s + e + m + p + t <= 64                       */
  int32_t exp_bias;       /* b_e of Sec. 2.3 (80 for e = 7, 127 for e = 8)     */
  int32_t map;            /* ivc_map                                           */
  int32_t underflow_mode; /* 0: below range -> lowest value (Sec. 2.3); 1: zero word */
  int32_t overflow_mode;  /* 0: saturate to the largest value; 1: infinite code */
  int32_t reserved;       /* must be 0                                         */
  double gamma;           /* IVC_MAP_TANH companding strength (paper: 0.5)     */
  int64_t nphi_max_p1;    /* IVC_MAP_FRACSPLIT: n_phi_max + 1                  */
} ivc_format;

/* Device-side event counters (device pointer; counts are added atomically). */
typedef struct {
  unsigned long long n_overflow, n_underflow, n_nonfinite;
} ivc_counts;

/* Fills *f with the paper's primary layout <0,7,22>-17-18, b7 = 80
 * (Sec. 3 and Sec. 5), uniform map, clamp below range, saturate above. */
ivc_status ivc_format_default(ivc_format *f);

/* IVC_OK if *f describes a supported format (field widths total <= 64,
 * theta_bits <= 20, phi_bits <= 19, fractional split within 2^40). */
ivc_status ivc_format_validate(const ivc_format *f);

/* Static text for a status code. */
const char *ivc_status_string(ivc_status s);

/* Library version string. */
const char *ivc_version(void);

/* ---------------------------------------------------------------------------
 * Compress n FP32 3-vectors into n words (Sec. 2.1 Eq. a_disc; Sec. 2.3;
 * Sec. 3).  xyz: device, layout per ivc_layout with leading dimension ld
 * (ignored for AoS).  w: device, n words.  counts: optional device pointer
 * (NULL to skip) receiving overflow / underflow / NaN counts.
 * Each word equals the exact-arithmetic encoding of the input, except where
 * the exact angle or magnitude lies within about 2^-40 of a rounding
 * boundary. */
ivc_status ivc_compress(const ivc_format *fmt, const float *xyz, ivc_layout layout,
                        int64_t ld, int64_t n, uint64_t *w, ivc_counts *counts,
                        ivc_stream_t stream);

/* Decompress n words (Eq. a_inv, Eq. cart2sphere): x = r cos(theta) sin(phi),
 * y = r sin(theta) sin(phi), z = r cos(phi), each component rounded away from
 * zero to FP32 (exact zeros are +0).  Non-finite words decode to NaN (or
 * infinities for the infinite code). */
ivc_status ivc_decompress(const ivc_format *fmt, const uint64_t *w, int64_t n,
                          float *xyz, ivc_layout layout, int64_t ld,
                          ivc_stream_t stream);

/* The same words as ivc_compress and the same vectors as ivc_decompress
 * (AoS layout only), with every rounding decision of Sec. 2.1 / Eq. a_disc
 * (angle bins), Sec. 2.3 (the RN32 magnitude) and Eq. a_inv (the decoded
 * components) taken by the exact-decision path in 64/128-bit integer
 * arithmetic that the fast kernels use only near a boundary: integer Taylor
 * series for cos/sin (about 2^-57 relative) and an exact norm decision.  No
 * floating point wider than FP32.  Slower; meant for validating results.
 * Arguments, ownership and errors as ivc_compress / ivc_decompress. */
ivc_status ivc_compress_exact(const ivc_format *fmt, const float *xyz, int64_t n, uint64_t *w,
                              ivc_counts *counts, ivc_stream_t stream);
ivc_status ivc_decompress_exact(const ivc_format *fmt, const uint64_t *w, int64_t n, float *xyz,
                                ivc_stream_t stream);

/* Sec. 5: c[i] = compress(decompress(a[i]) + decompress(b[i])), FP32 adds. */
ivc_status ivc_add(const ivc_format *fmt, const uint64_t *a, const uint64_t *b,
                   uint64_t *c, int64_t n, ivc_stream_t stream);

/* y[i] = compress(fmaf(alpha, decompress(x[i]), decompress(y[i]))).
 * The paper's Sec. 5 kernel (decompress both operands, combine in FP32,
 * compress the result) with the combination y + alpha x in place of a + b,
 * one fused multiply-add per component (single rounding).  In place: y is
 * read and written.  Words: device, 8-byte aligned (16 for the two-per-thread
 * kernel).  Errors and results as ivc_add. */
ivc_status ivc_axpy(const ivc_format *fmt, float alpha, const uint64_t *x,
                    uint64_t *y, int64_t n, ivc_stream_t stream);

/* Pointwise update of a compressed field (velocity v, forcing f):
 * v_new = fmaf(dt, decompress(f[i]), decompress(v[i]));
 * v_out[i] = compress(v_new); if rho and m_out are both non-NULL,
 * m_out[i] = compress(rho[i] * v_new) (FP32 products).  rho: device FP32.
 * The Sec. 5 pattern (decompress, FP32 arithmetic, recompress) applied to the
 * flow variables the paper compresses in its test cases: the velocity and
 * momentum 3-vectors of the Taylor-Green vortex of Sec. 4.2 (initial fields
 * there), advanced by an explicit forcing step.  v_out may equal v (in place);
 * m_out must not alias v, f or v_out.  Errors as ivc_add. */
ivc_status ivc_pointwise_update(const ivc_format *fmt, float dt, const uint64_t *v,
                                const uint64_t *f, const float *rho, uint64_t *v_out,
                                uint64_t *m_out, int64_t n, ivc_stream_t stream);

/* ---------------------------------------------------------------------------
 * Uncompressed baselines (the paper's C = A + B on 3 x N FP32, Sec. 5), for
 * the same operations on plain storage.  FP32: layout AoS or SoA (ld as
 * above).  FP16 / BF16: AoS, elements as raw uint16_t bits; arithmetic in
 * FP32, results rounded to nearest even. */
ivc_status ivc_f32_add(ivc_layout layout, const float *a, const float *b, float *c,
                       int64_t ld, int64_t n, ivc_stream_t stream);
ivc_status ivc_f32_axpy(ivc_layout layout, float alpha, const float *x, float *y,
                        int64_t ld, int64_t n, ivc_stream_t stream);

typedef enum { IVC_F16 = 0, IVC_BF16 = 1 } ivc_half_kind;
ivc_status ivc_half_add(ivc_half_kind kind, const uint16_t *a, const uint16_t *b,
                        uint16_t *c, int64_t n, ivc_stream_t stream);
ivc_status ivc_half_axpy(ivc_half_kind kind, float alpha, const uint16_t *x,
                         uint16_t *y, int64_t n, ivc_stream_t stream);
/* FP32 AoS <-> FP16/BF16 AoS conversion of n 3-vectors (round to nearest even). */
ivc_status ivc_half_from_f32(ivc_half_kind kind, const float *xyz, uint16_t *h,
                             int64_t n, ivc_stream_t stream);
ivc_status ivc_half_to_f32(ivc_half_kind kind, const uint16_t *h, float *xyz,
                           int64_t n, ivc_stream_t stream);

/* ---------------------------------------------------------------------------
 * Error statistics of stored vectors against FP32 originals (Eq. stat and the
 * normalised errors of Sec. 3), reduced in FP64 on the device.  x, xh: device
 * AoS FP32, n vectors; vectors with a zero or non-finite original are skipped.
 * out: device, IVC_STATS_LEN doubles, ACCUMULATED into (zero it first):
 *   [0] count   [1] sum e   [2] sum e^2   [3] max e
 *   [4] sum e/|x|   [5] max e/|x|
 *   [6] sum ang^2   [7] max ang            (angle between x and xh, radians)
 *   [8] sum rel^2   [9] max rel            (rel = ||xh| - |x|| / |x|)
 *   [10] count of xh non-finite where x is finite                         */
#define IVC_STATS_LEN 11
ivc_status ivc_error_stats(const float *x, const float *xh, int64_t n, double *out,
                           ivc_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batched form over many fields of uneven length (one persistent launch
 * driven by a device work list, replayed from a CUDA graph).  There is no
 * counterpart in the paper: it is a library-level way to run the Sec. 5 add
 * and the axpy above over many fields at once (the fields of a
 * multi-partition mesh, each with its own length), with results identical to
 * one ivc_add / ivc_axpy call per field. */
typedef enum { IVC_OP_ADD = 0, IVC_OP_AXPY = 1 } ivc_op;

typedef struct {
  const uint64_t *a;  /* add: first operand;  axpy: x                 */
  const uint64_t *b;  /* add: second operand; axpy: unused (NULL)      */
  uint64_t *c;        /* add: result;         axpy: y (in/out)         */
  int64_t n;          /* vectors in this field (>= 0)                  */
  float alpha;        /* axpy scale                                    */
  float reserved;
} ivc_field;

/* Launch shape picked by ivc_tune (or given by the caller). */
typedef struct {
  int32_t block;         /* threads per block (64 .. 1024, multiple of 32) */
  int32_t vec_per_thread;/* vectors per thread per step: 1, 2 or 4          */
  int32_t tile;          /* vectors per work-list tile (batched form)       */
  int32_t blocks_per_sm; /* resident blocks per SM for persistent grids     */
} ivc_launch_config;

typedef struct ivc_plan_s *ivc_plan;

/* Builds a plan for `nfields` fields.  The field table and the work list are
 * written into the caller's device `workspace`; call first with
 * workspace == NULL to get the required size in *ws_bytes.  cfg may be NULL
 * (default shape).  The plan captures one launch (counter reset + persistent
 * kernel) in a CUDA graph on `stream`.  The field descriptors are copied;
 * the data pointers must stay valid while the plan is used. */
ivc_status ivc_plan_batched(const ivc_format *fmt, ivc_op op, const ivc_field *fields,
                            int nfields, void *workspace, size_t *ws_bytes,
                            const ivc_launch_config *cfg, ivc_stream_t stream,
                            ivc_plan *plan);
/* Replays the plan's graph on `stream`. */
ivc_status ivc_launch_plan(ivc_plan plan, ivc_stream_t stream);
/* Same work as ivc_launch_plan, as one ordinary persistent launch (no graph). */
ivc_status ivc_launch_plan_direct(ivc_plan plan, ivc_stream_t stream);
/* Device status word of the plan's last launch: IVC_OK, or IVC_ERR_TIMEOUT
 * if the bounded scheduling loop ran out.  Synchronises `stream`. */
ivc_status ivc_plan_status(ivc_plan plan, ivc_stream_t stream);
ivc_status ivc_plan_destroy(ivc_plan plan);

/* Launch-shape tuner (no counterpart in the paper; results do not depend on
 * the shape).  Times candidate launch shapes of `op` on the caller's buffers (n vectors;
 * for IVC_OP_AXPY, b is used as the y operand and is overwritten; for
 * IVC_OP_ADD, c is overwritten) and writes the fastest to *best.  Runs
 * synchronously on `stream`. */
ivc_status ivc_tune(const ivc_format *fmt, ivc_op op, const uint64_t *a, const uint64_t *b,
                    uint64_t *c, int64_t n, ivc_stream_t stream, ivc_launch_config *best);

/* Autotuner of the batched form (no counterpart in the paper; results do
 * not depend on the shape): builds plans for candidate shapes -- block size
 * (128, 256), resident blocks per SM (1, 2, ... up to the occupancy limit)
 * and work-list tile (2048 ... 131072 vectors) -- in the caller's workspace
 * (ws_bytes as sized by ivc_plan_batched), times each with ordinary
 * persistent launches on `stream` (the fields' outputs are overwritten) and
 * writes the fastest to *best (vec_per_thread reports the kernel's vectors
 * per thread per step: 2 on the packed fast path, else 1).  Synchronous. */
ivc_status ivc_tune_batched(const ivc_format *fmt, ivc_op op, const ivc_field *fields,
                            int nfields, void *workspace, size_t ws_bytes, ivc_stream_t stream,
                            ivc_launch_config *best);

/* Add with an explicit launch shape (cfg NULL = default). */
ivc_status ivc_add_cfg(const ivc_format *fmt, const uint64_t *a, const uint64_t *b,
                       uint64_t *c, int64_t n, const ivc_launch_config *cfg,
                       ivc_stream_t stream);

/* Random-access decompression (the unstructured access the method is meant
 * for, Sec. 1): xyz[3i .. 3i+2] = decompress(w[idx[i]]) for 0 <= i < n, with
 * the decode of Sec. 2.1 / Eq. a_inv (results as ivc_decompress).
 *   w    device words, nw of them (8-byte aligned; may be NULL when nw == 0).
 *   idx  device int64 indices (8-byte aligned; 16-byte aligned with an
 *        8-byte aligned xyz selects the two-per-thread kernel).
 *   xyz  device FP32 output, AoS, 3 n floats.
 * An index outside [0, nw) reads nothing and gives NaN components.
 * Errors: IVC_ERR_ARG (n < 0, nw < 0, NULL pointers), IVC_ERR_ALIGN. */
ivc_status ivc_gather_decompress(const ivc_format *fmt, const uint64_t *w, int64_t nw,
                                 const int64_t *idx, int64_t n, float *xyz,
                                 ivc_stream_t stream);

/* The FP32 baseline of ivc_gather_decompress: out[3i .. 3i+2] = the vector
 * src[idx[i]] of an AoS source (3 floats per vector) or an SoA source (rows x,
 * y, z at stride ld >= nsrc).  Out-of-range indices give NaN components. */
ivc_status ivc_f32_gather(ivc_layout layout, const float *src, int64_t ld, int64_t nsrc,
                          const int64_t *idx, int64_t n, float *out, ivc_stream_t stream);

/* Divergence of a compressed flux: Algorithm 1 (Sec. 4; Table fr_nse, step
 * 10) of the flux-reconstruction right-hand side.  For every element e and
 * solution point k, and every equation p:
 *     div(k, p, e) = sum_j sum_c D[c ns + j][k] * X(j, p, e)_c
 * where X(j, p, e) = decompress(F(j, p, e)) is the 3-vector flux row of
 * equation p at point j of element e (Sec. 2), and D the element's divergence
 * operator.  Products and sums in FP32, order unspecified (error within the
 * FP32 summation bound of the 3 ns terms).
 *   F    device words, row (j, p) of element e at F[(j * nvars + p) * ld + e]
 *        (element index fastest, ld >= ne).
 *   D    device FP32, row-major (3 ns) x ns: D[(c * ns + j) * ns + k] is the
 *        derivative along axis c (0, 1, 2 = x, y, z) of the basis function of
 *        point j, evaluated at point k.
 *   div  device FP32 output, (k, p, e) at div[(k * nvars + p) * ld_out + e],
 *        ld_out >= ne; entries with e >= ne are not written.
 * Limits: 1 <= ns <= 64 (hex elements up to degree 3), 1 <= nvars <= 5.
 * Errors: IVC_ERR_ARG for sizes out of range or NULL pointers with ne > 0,
 * IVC_ERR_ALIGN for F not 8-byte or D / div not 4-byte aligned.
 * The products run on the tensor cores (tcgen05, FP32 accumulation, each FP32
 * operand split into a TF32 head and tail: three TF32 products per term, the
 * result within the FP32 summation bound above). */
ivc_status ivc_flux_divergence(const ivc_format *fmt, const uint64_t *F, int64_t ld, int ns,
                               int nvars, int64_t ne, const float *D, float *div,
                               int64_t ld_out, ivc_stream_t stream);

/* The same divergence with FP32 FMAs on the CUDA cores (a block of decoding
 * warps and FMA warps handing buffers over through mbarriers), kept for
 * comparison; same arguments, limits and errors. */
ivc_status ivc_flux_divergence_simt(const ivc_format *fmt, const uint64_t *F, int64_t ld, int ns,
                                    int nvars, int64_t ne, const float *D, float *div,
                                    int64_t ld_out, ivc_stream_t stream);

/* Bound, in SM clock cycles, of every wait between the decoding and the
 * accumulating warps of the CUDA-core kernel (ivc_flux_divergence_simt,
 * ivc_f32_flux_divergence_simt) launched after this call; cycles <= 0
 * restores the default (2e9, about a second).  A wait that runs out ends the
 * block (its copies completed first) and makes the next
 * ivc_flux_divergence_check return IVC_ERR_TIMEOUT; the output of that launch
 * is undefined.  Meant for testing that failure path; host state, not
 * thread-safe against concurrent launches. */
ivc_status ivc_set_flux_divergence_wait_limit(long long cycles);

/* Reports (and clears) a failure of the flux-divergence kernels since the
 * last check: their decoding and accumulating warps hand shared-memory
 * buffers to each other through barriers whose waits are bounded (about a
 * second); a wait that runs out ends the launch early and is reported here as
 * IVC_ERR_TIMEOUT.  Synchronises with the current device.  IVC_OK otherwise. */
ivc_status ivc_flux_divergence_check(void);

/* The same divergence from an uncompressed FP32 flux (the baseline of
 * Algorithm 1): component c of row (j, p) of element e at
 * F[((c * ns + j) * nvars + p) * ld + e].  Other arguments as above. */
ivc_status ivc_f32_flux_divergence(const float *F, int64_t ld, int ns, int nvars, int64_t ne,
                                   const float *D, float *div, int64_t ld_out,
                                   ivc_stream_t stream);
/* ... and its CUDA-core counterpart. */
ivc_status ivc_f32_flux_divergence_simt(const float *F, int64_t ld, int ns, int nvars,
                                        int64_t ne, const float *D, float *div, int64_t ld_out,
                                        ivc_stream_t stream);

/* The compressed add c = a + b (Sec. 5) of HOST-resident words: a, b, c are
 * host pointers.  When all three are page-locked (cudaHostAlloc or
 * registered), the kernel reads and writes them directly over the host link
 * on `stream` and the workspace is not used (may be NULL).  Otherwise the
 * words stream through the caller's device `workspace` (16-byte aligned,
 * ws_bytes long) in chunks of floor(ws_bytes / 72) & ~1 vectors, three chunks
 * in flight on streams of the library's own, so that host-to-device copies,
 * kernels and device-to-host copies of consecutive chunks overlap.  The work
 * starts after what is already queued on `stream`, and `stream` waits for all
 * of it: the host buffers and the workspace must stay valid until `stream`
 * completes.  Results are those of ivc_add.  Errors: IVC_ERR_ARG (NULL
 * pointers, n < 0, no workspace for pageable memory), IVC_ERR_ALIGN (host
 * pointers not 8-byte, workspace not 16-byte aligned), IVC_ERR_NOMEM
 * (workspace below 144 bytes), IVC_ERR_CUDA; on an error, chunks already
 * queued may still run. */
ivc_status ivc_add_host(const ivc_format *fmt, const uint64_t *a, const uint64_t *b,
                        uint64_t *c, int64_t n, void *workspace, size_t ws_bytes,
                        ivc_stream_t stream);

/* ------------------------------------------------------------------------
 * Flux-reconstruction steps 5-11 of Table fr_nse (Sec. 4) with compressed
 * tensor rows.  Higher-dimensional terms (gradients, metric terms, normals,
 * fluxes) are compressed row by row (Eq. eulerF): every row is one 3-vector,
 * one 64-bit word.  Step 10 is ivc_flux_divergence.  Each step has an FP32
 * counterpart (ivc_f32_fr_*) with the same arithmetic on uncompressed rows.
 *
 * Elements are hexahedra of degree k = order (1..3) with q = k + 1
 * Gauss-Legendre points per axis: ns = q^3 solution points, j = (jz q + jy) q
 * + jx, and nf = 6 q^2 flux points, f = (2 c + s) q^2 + b q + a on the face of
 * axis c (0, 1, 2 = x, y, z) and side s (0 at xi_c = -1, 1 at +1), with a, b
 * the indices along the other two axes in increasing order.
 *
 * Layout (element index e fastest; one leading dimension ld >= ne for every
 * array of a call): a scalar of point k and variable v at [(k nv + v) ld + e];
 * a compressed row at the same index of a uint64_t array; an FP32 row with
 * component c at [((c npts + k) nv + v) ld + e] (npts = ns or nf).  Metric
 * rows use nv = 3 (the rows of S = |J| J^-1, J = dx/dxi), normals nv = 1.
 * Entries with e >= ne are neither read nor written.  The caller owns every
 * buffer (device memory); unless stated, inputs and outputs must not overlap.
 * Arithmetic is FP32 on the decoded rows; compressed outputs are encoded as
 * ivc_compress does.
 * Errors: IVC_ERR_ARG (order outside 1..3, nvars outside 1..5, ne < 0,
 * ld < ne, NULL pointers with ne > 0, mesh dims whose product is not ne),
 * IVC_ERR_ALIGN (words not 8-byte, floats not 4-byte aligned), IVC_ERR_FORMAT.
 * ------------------------------------------------------------------------ */

/* The one-dimensional basis on the q Gauss-Legendre points xi_i of [-1, 1]. */
typedef struct {
  int order;          /* k, 1..3 */
  float dm[16];       /* dm[i * q + a] = l_a'(xi_i), derivative of basis function a */
  float lm[4], lp[4]; /* l_a(-1), l_a(+1): interpolation to the ends */
  float gl[4], gr[4]; /* g_L'(xi_i), g_R'(xi_i): derivatives of the correction functions */
} ivc_fr_basis;

/* Constant-property gas: ratio of specific heats, dynamic viscosity, Prandtl
 * number (heat flux kappa grad T = mu gamma / ((gamma - 1) Pr) grad(p / rho)). */
typedef struct {
  float gamma, mu, prandtl;
} ivc_fr_gas;

/* Step 5: grad(k, v) = sum_a dm[k_c][a] w(point k with k_c = a, v) along each
 * axis c: the reference-space gradient rows of the nvars scalars w (the
 * primitives) at the solution points. */
ivc_status ivc_fr_gradient(const ivc_format *fmt, const ivc_fr_basis *basis, const float *w,
                           int64_t ne, int64_t ld, int nvars, uint64_t *grad,
                           ivc_stream_t stream);
ivc_status ivc_f32_fr_gradient(const ivc_fr_basis *basis, const float *w, int64_t ne,
                               int64_t ld, int nvars, float *grad, ivc_stream_t stream);

/* Step 6: grad_c(k, v)_c = grad(k, v)_c + gl[k_c] dw(f_L, v) + gr[k_c] dw(f_R, v)
 * with f_L, f_R the flux points of the two faces of axis c on the line of k
 * and dw the interface jumps (w^I - w^f) at the flux points (scalars, nf
 * points).  grad_c may equal grad (in place). */
ivc_status ivc_fr_correct_gradient(const ivc_format *fmt, const ivc_fr_basis *basis,
                                   const uint64_t *grad, const float *dw, int64_t ne, int64_t ld,
                                   int nvars, uint64_t *grad_c, ivc_stream_t stream);
ivc_status ivc_f32_fr_correct_gradient(const ivc_fr_basis *basis, const float *grad,
                                       const float *dw, int64_t ne, int64_t ld, int nvars,
                                       float *grad_c, ivc_stream_t stream);

/* Step 7: rows at the flux points, rows_f(f, v) = sum_i l_i(-1 or +1) rows(point
 * i along the face's axis on the line of f, v). */
ivc_status ivc_fr_interp_rows(const ivc_format *fmt, const ivc_fr_basis *basis,
                              const uint64_t *rows, int64_t ne, int64_t ld, int nvars,
                              uint64_t *rows_f, ivc_stream_t stream);
ivc_status ivc_f32_fr_interp_rows(const ivc_fr_basis *basis, const float *rows, int64_t ne,
                                  int64_t ld, int nvars, float *rows_f, ivc_stream_t stream);

/* Step 8: out(f, v) = nFinv(f, v) - n(f) . F_vis^I(f, v) at every flux point
 * of every element of a periodic dims[0] x dims[1] x dims[2] mesh (ne = the
 * product, e = (ez dims[1] + ey) dims[0] + ex), with the BR1 common viscous
 * flux F_vis^I = (F_vis(this side) + F_vis(partner)) / 2; the partner is the
 * point with the same (a, b) on the facing face of the neighbouring element.
 * F_vis is the compressible Navier-Stokes viscous flux (Stokes hypothesis) of
 * the conserved q_f (5 scalars) and the physical gradient (S^T grad_f) / |J|
 * of the primitives (rho, u, v, w, p) from their reference gradient rows
 * grad_f (5 rows), the metric rows S_f (3 rows) and detJ_f = |J|.  nrm: one
 * row per flux point, this side's scaled normal.  nvars = 5. */
ivc_status ivc_fr_common_viscous_flux(const ivc_format *fmt, int order, const ivc_fr_gas *gas,
                                      const int dims[3], const uint64_t *grad_f,
                                      const uint64_t *nrm, const uint64_t *S_f,
                                      const float *detJ_f, const float *q_f, const float *nFinv,
                                      int64_t ld, float *out, ivc_stream_t stream);
ivc_status ivc_f32_fr_common_viscous_flux(int order, const ivc_fr_gas *gas, const int dims[3],
                                          const float *grad_f, const float *nrm,
                                          const float *S_f, const float *detJ_f,
                                          const float *q_f, const float *nFinv, int64_t ld,
                                          float *out, ivc_stream_t stream);

/* Step 9: the reference flux rows F(k, v) = S (F_inv - F_vis) at the solution
 * points from the conserved q_s (5 scalars), the primitives' reference
 * gradient rows grad (5 rows), the metric rows S_s (3 rows) and detJ_s; the
 * rows of F_inv are those of Eq. eulerF.  nvars = 5. */
ivc_status ivc_fr_flux(const ivc_format *fmt, int order, const ivc_fr_gas *gas, const float *q_s,
                       const uint64_t *grad, const uint64_t *S_s, const float *detJ_s,
                       int64_t ne, int64_t ld, uint64_t *F, ivc_stream_t stream);
ivc_status ivc_f32_fr_flux(int order, const ivc_fr_gas *gas, const float *q_s, const float *grad,
                           const float *S_s, const float *detJ_s, int64_t ne, int64_t ld,
                           float *F, ivc_stream_t stream);

/* Step 11: Fc(f, v) = nF(f, v) - sign(s) (row F interpolated to f)_c: the
 * interface flux minus the interior normal flux (scalars at the flux points). */
ivc_status ivc_fr_flux_correction(const ivc_format *fmt, const ivc_fr_basis *basis,
                                  const uint64_t *F, const float *nF, int64_t ne, int64_t ld,
                                  int nvars, float *Fc, ivc_stream_t stream);
ivc_status ivc_f32_fr_flux_correction(const ivc_fr_basis *basis, const float *F, const float *nF,
                                      int64_t ne, int64_t ld, int nvars, float *Fc,
                                      ivc_stream_t stream);

/* Frees the cached per-format tables on the current device. */
ivc_status ivc_release_tables(void);

/* Same result as ivc_add, for callers that must not allocate device memory
 * (for example code running under a framework whose caching allocator owns
 * the device memory, or a latency-critical loop that cannot afford
 * cudaMalloc's implicit synchronisation).  There is no counterpart in the
 * paper: this is a library-level variant of the compressed add.
 * The tables live in a fixed 32 KiB device array inside the library (held by
 * every GPU that loads it until exit) instead of cudaMalloc'd memory.  The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and it keeps the last call's contents; a call
 * with a format whose tables are not the ones the array holds first copies
 * them (host-built, the values ivc_add uses) on `stream` and records an event;
 * every later call on any stream waits for that event before its kernel.
 * Calls that overlap on the GPU with different formats race on the array.
 * While `stream` is capturing, the first call on a device and a call that
 * would rewrite the tables return IVC_ERR_UNSUPPORTED; a captured call reads
 * the array when the graph runs, so a later call with another format changes
 * what a replay of that graph decodes with.  Calls no cudaMalloc/cudaFree.
 * Errors: as ivc_add, plus IVC_ERR_UNSUPPORTED for the tanh map and
 * IVC_ERR_NOMEM for a format whose tables exceed the array (more than 2048
 * entries). */
ivc_status ivc_add_noalloc(const ivc_format *fmt, const uint64_t *a, const uint64_t *b,
                           uint64_t *c, int64_t n, ivc_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* IVC_H */

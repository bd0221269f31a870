/*
 * fq.h -- exact dense matrix products over small finite fields on GB300 (sm_103a).
 *
 * Boothby & Bradshaw, "Bitslicing and the Method of Four Russians Over Larger
 * Finite Fields".  Matrices are stored bitsliced (Section 3): bit i of every
 * element's code lives in bit-plane i, 64 elements per 64-bit word.  Products use
 * the Method of Four Russians with an additive basis (Section 2).
 *
 * Fields (argument q):
 *   q = 2  F_2,  1 plane, the element itself (Section 2's binary case), basis {1};
 *   q = 3  F_3,  2 planes, codes (x0, x1): 0 = (0,0), 1 = (1,0), -1 = (1,1)
 *          (Section 4.1), additive basis {1, -1};
 *   q = 5  F_5,  3 planes, binary digits of the residue (Section 4.2), basis {1,2,4};
 *   q = 7  F_7,  3 planes, binary digits of the residue (Section 4.2), basis {1,2,4};
 *   q = 4  GF(4) = F_2[x]/(x^2+x+1), 2 planes, element a0 + alpha*a1 has code
 *          a0 + 2*a1 (Section 4.3), basis {1, alpha};
 *   q = 8, 9, 25, 27, 49, 125: the extension fields F_{p^n} = F_p[x]/(f) of
 *          Section 4.3 ("non-prime fields"), with f = x^3 + x + 1, x^2 + 2x + 2,
 *          x^2 + 4x + 2, x^3 + 2x + 1, x^2 + 6x + 3, x^3 + 3x + 3 (monic,
 *          irreducible and primitive).  Element c_0 + c_1 x + ... has code
 *          sum_j c_j p^j; a matrix is stored as its coefficient matrices
 *          A = A_0 + A_1 x + ..., the planes of A_0 (as an F_p matrix), then
 *          those of A_1, ... -- n * fq_planes(p) planes.  GF(4) is the same
 *          layout for p = 2, n = 2.  Products are Section 4.3's matrix-level
 *          products: Karatsuba (3 base-field products) for n = 2, the paper's
 *          trinomial formula (6 products) for n = 3, then reduction by f.
 *
 * Packed layout ("planes buffer") of a rows x cols matrix: plane-major,
 *   word(p, r, w) = buf[(p * rows + r) * pitch + w],  pitch = fq_pitch_words(cols),
 * element c of row r is bit (c mod 64) of word floor(c / 64) of each plane.
 * Words past the last column (padding) must be zero in inputs and are zero in
 * outputs; fq_pack writes them.  Planes buffers must be 16-byte aligned device
 * memory (cudaMalloc and PyTorch allocations are).  Output codes are canonical
 * (F_5 and F_7 codes are reduced to [0, p)).
 *
 * Conventions: every function is asynchronous on `stream` (a cudaStream_t, or
 * NULL for the legacy default stream) unless it says otherwise; the caller owns
 * all device buffers; argument errors are returned before anything is
 * enqueued.  Errors a kernel detects while running (a residue >= q in fq_pack, a
 * bounded device wait that gave up) are recorded on the device and returned by
 * fq_status().
 *
 * Debug build: compiled with -DFQ_DEBUG (libfq_gb300_debug.so, same ABI), the
 * kernels also check every table index of a Four-Russians lookup against the
 * table (idx < 2^k) and every store of C against its rows and row pitch; a
 * failed check records FQ_EBOUNDS and the access is skipped (or made to entry
 * 0 of the table).  The release library has no such checks.
 */
#ifndef FQ_H
#define FQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define FQ_OK 0
#define FQ_EINVAL 1    /* bad q, shape, pointer, alignment or option              */
#define FQ_EVALUE 2    /* a residue >= q was passed to fq_pack (device-detected)   */
#define FQ_ECUDA 3     /* a CUDA call failed; see fq_last_cuda_error()            */
#define FQ_ETIMEOUT 4  /* a bounded device wait gave up (device-detected)          */
#define FQ_ENOTSUP 5   /* valid request the library does not support              */
#define FQ_ENOMEM 6    /* host allocation failed                                   */
#define FQ_EBOUNDS 7   /* a bounds check of the FQ_DEBUG build failed (device-detected) */

/* ---- product paths (fq_options.path) --------------------------------------- */
#define FQ_PATH_AUTO 0 /* planner's choice                                         */
#define FQ_PATH_M4RM 1 /* bitsliced Method of Four Russians (Sections 2-4)         */
#define FQ_PATH_MMA 2  /* exact tensor-core contraction (tcgen05; mma.sync s8 for long l) */
#define FQ_PATH_KARATSUBA 3 /* GF(4) only: Section 4.3's three F_2 products        */

/* Number of bit-planes of a field element (1 for q = 2; 2 for q = 3, 4; 3 for
 * q = 5, 7; n * fq_planes(p) for q = p^n), or 0 for an unsupported q.  Section 4
 * fixes the widths. */
int fq_planes(int q);

/* Row pitch in 64-bit words of a planes buffer with `cols` columns:
 * ceil(cols / 64) rounded up to a multiple of 16 (128 bytes).  -1 if cols < 0. */
int64_t fq_pitch_words(int64_t cols);

/* Total 64-bit words of a planes buffer: fq_planes(q) * rows * fq_pitch_words(cols);
 * -1 on bad arguments. */
int64_t fq_planes_words(int q, int64_t rows, int64_t cols);

/* Pack residues (element codes) into bit-planes (Section 3; codes of Sections
 * 4.1-4.3).
 * res:    device, rows x cols uint8 codes in [0, q), row-major, leading
 *         dimension ld >= cols (elements).
 * planes: device planes buffer (layout above), written entirely, padding zeroed.
 * A residue >= q is stored as 0 and recorded for fq_status() (FQ_EVALUE). */
int fq_pack(int q, int64_t rows, int64_t cols, const uint8_t *res, int64_t ld,
            uint64_t *planes, void *stream);

/* Unpack bit-planes into residues in [0, q).  Any 3-bit code is accepted for
 * F_5/F_7 and read mod p (codes are not unique, Section 4.2).
 * planes: device planes buffer; res: device rows x cols uint8, leading dim ld. */
int fq_unpack(int q, int64_t rows, int64_t cols, const uint64_t *planes,
              uint8_t *res, int64_t ld, void *stream);

/* Elementwise Z = X + Y (sub = 0) or Z = X - Y (sub = 1) of packed matrices with
 * the bitsliced formulas of Sections 4.1-4.3 -- the row additions the product is
 * built from.  X, Y, Z: device planes buffers of the same shape (Z may alias X or
 * Y).  F_5/F_7 outputs may be non-canonical codes (fq_unpack reduces them). */
int fq_add(int q, int64_t rows, int64_t cols, const uint64_t *X, const uint64_t *Y,
           uint64_t *Z, int sub, void *stream);

/* Options for fq_matmul_ex; zero-initialise for defaults. */
typedef struct fq_options {
  int path;      /* FQ_PATH_*; for q = 8 .. 125 the base-field products' path      */
  int k;         /* M4RM block size: 0 = planner, else 6..10 (Section 2's k)       */
  int64_t chunk; /* MMA path: l-chunk length between mod-p reductions; 0 = largest */
  int variant;   /* M4RM rows per CTA: 0 = planner, else 1 .. the kernel's maximum;
                    tcgen05 path: row blocks per group of the tile order (0 = 8,
                    16 for the fp4 form)                                     */
  int kernel;    /* M4RM kernel: 0 = planner, i + 1 = compiled kernel i of field q;
                    tensor-core path: 0 = tcgen05 by shape, 1 = the mma.sync
                    s8 form, 2 = tcgen05 on single SMs (128 x 256 tiles),
                    3 = on SM pairs (256 x 256), 4 = on SM pairs (256 x 512),
                    all three from e4m3 operands; 5 = on SM pairs (256 x 448)
                    from packed e2m1 operands (kind::mxf4)                  */
  int strassen;  /* Strassen-Winograd levels over the base-field products: 0 = the
                    time model decides, -1 = none, L > 0 = L levels (each needs
                    m, l, n to be multiples of 2048 at that level)               */
  int reserved[3];
} fq_options;

/* C = A B over F_q (Section 2: C_i = sum_s sum_d alpha_d T_s[phi_d(A_i, block s)]).
 * A: device planes buffer m x l; B: l x n; C: m x n (written entirely; must not
 * alias A or B).  m, l, n >= 0; l = 0 gives C = 0.  The product is exact.
 * Extension fields (q = 8 .. 125, and GF(4) with FQ_PATH_KARATSUBA) run
 * Section 4.3's matrix-level product: the base-field operand sums with fq_add's
 * formulas, 3 or 6 base-field products (each on fq_options.path: AUTO, M4RM or
 * MMA; k, variant and kernel refer to the base field's kernels) and one
 * elementwise combination kernel.  Their scratch (the operand sums and the
 * products beyond n, about (3 or 6 - n) x the base-field size of A, B and C)
 * is stream-ordered on `stream` (a CUDA graph capture records it as
 * allocation nodes) from the library's own memory pool on the device. */
int fq_matmul(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A,
              const uint64_t *B, uint64_t *C, void *stream);

/* fq_matmul with explicit options (path, k, l-chunk, tile variant, Strassen
 * levels); opt may be NULL.
 *
 * Strassen-Winograd (the paper's remark that M4RM serves as the base case of an
 * asymptotically faster product, Section 2): one level computes C from seven
 * half-size products and fifteen bitsliced additions over quadrants, which are
 * copied out of and back into the packed matrices.  Levels need m, l, n to be
 * multiples of 2048 (halves of whole 1024-column pitches); with strassen = 0 a
 * level is taken only where the time model expects seven half-size products
 * and the additions to beat the direct product (on GB300, F_3 from 16384 on).
 * Scratch (the quadrants, eight operand sums and seven products, about 3.4x
 * the size of A, B and C together at the top level) is stream-ordered on
 * `stream` from the library's own memory pool, see fq_release_scratch. */
int fq_matmul_ex(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A,
                 const uint64_t *B, uint64_t *C, void *stream, const fq_options *opt);

/* The number of Strassen-Winograd levels fq_matmul_ex takes for (q, m, l, n)
 * with these options (opt may be NULL) on the current device: >= 0, or
 * -FQ_EINVAL / -FQ_ECUDA.  Host-only apart from the device attribute query. */
int fq_strassen_levels(int q, int64_t m, int64_t l, int64_t n, const fq_options *opt);

/* ---- the tensor-core path in two stages -------------------------------------
 * FQ_PATH_MMA runs on the tcgen05 tensor cores whenever l * ((p-1)/2)^2 < 2^24
 * (l < 2^24 for GF(4)), in one of two operand formats:
 *   - kind::f8f6f4 with e4m3 operands (forms 2, 3, 4: single SMs, SM pairs
 *     with 256 x 256 tiles, SM pairs with 256 x 512 tiles);
 *   - kind::mxf4 with packed e2m1 operands, two to a byte, every block scale
 *     factor 1.0 (form 5: SM pairs, 256 x 448 tiles), at twice the e4m3 rate.
 * Both accumulate in fp32.  The balanced residues 0, +-1, +-2, +-3 are exact
 * in e4m3 and in e2m1, and every partial sum is an integer below 2^24, so the
 * sums are exact and the product is bit-exact.  By shape, products of at most
 * 128 rows take form 2, products of more rows and l >= 2048 form 5, the rest
 * form 3 (fq_tc_form); fq_options.kernel = 2 .. 5 forces a form.  Longer l, or
 * fq_options.chunk > 0, or fq_options.kernel = 1 select the mma.sync s8 form
 * with mod-p reduction every chunk.  fq_matmul converts the operands into
 * stream-ordered scratch; these calls expose the two stages (in the shape's
 * default form) so that a caller can keep the converted operands:
 *   fq_tc_form: the form (2 .. 5) the shape takes, or -FQ_ENOTSUP outside the
 *     tcgen05 path's range, -FQ_EINVAL for a bad q or size.  Host-only;
 *   fq_tc_workspace_bytes: device bytes of the converted operands, or -1
 *     outside the tcgen05 form (bad q, negative size, l too long).  Forms 2, 3,
 *     4: A as m x la e4m3 bytes, B transposed as 64 * fq_pitch_words(n) x la,
 *     la = l rounded up to 128.  Form 5: A as m rows and B transposed as
 *     64 * fq_pitch_words(n) rows of la / 2 bytes, la = l rounded up to 256.
 *     Three such pairs for GF(4), whose product is three F_2 products by
 *     Section 4.3's Karatsuba form;
 *   fq_tc_prepare: A, B (planes buffers) -> workspace (16-byte aligned);
 *   fq_tc_multiply: workspace -> C (planes buffer, written entirely).
 * Both are asynchronous on `stream`; FQ_ENOTSUP outside the tcgen05 form. */
int fq_tc_form(int q, int64_t m, int64_t l, int64_t n);
int64_t fq_tc_workspace_bytes(int q, int64_t m, int64_t l, int64_t n);
int fq_tc_prepare(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B,
                  void *workspace, void *stream);
int fq_tc_multiply(int q, int64_t m, int64_t l, int64_t n, const void *workspace, uint64_t *C,
                   void *stream);

/* ---- many products in one launch ------------------------------------------
 * A plan assigns each of `count` products C_p = A_p B_p (shapes m[p] x l[p]
 * times l[p] x n[p], all over the same field q) to one of the two paths by
 * their time models (or as the caller asks):
 *   - Four Russians: work items (rows x a column tile of one product) with a
 *     block size k chosen per item by the planner's cost model, longest first;
 *   - tcgen05 (F_3, F_5, F_7 with 0 < l within the exact range and
 *     n <= 2^30): whole products are given to 76 groups of two persistent
 *     CTAs (one thread-block cluster each; longest first, each to the
 *     least-loaded group by the model; a group then takes its products
 *     smallest first).  A group's converter warps write each product's A
 *     and B as e4m3 bytes into one of the group's two scratch buffers in
 *     the workspace while its tensor-core warps compute the previous
 *     product's 128 x 256 tiles from the other, the two CTAs taking
 *     alternate tiles.  A product runs on two SMs: a batch of a few very
 *     large products is better served by fq_matmul.
 * The plan is host memory owned by the library. */
typedef struct fq_batch_plan fq_batch_plan;

/* Build a plan (host only).  q = 3, 4, 5 or 7.  m, l, n: host arrays of `count`
 * sizes (each >= 0 and < 2^31).  path: FQ_PATH_AUTO (per-product choice by the
 * models), FQ_PATH_M4RM (every product by Four Russians) or FQ_PATH_MMA (every
 * product the tcgen05 form can take; GF(4) and the rest by Four Russians);
 * fq_batched_plan_create is path FQ_PATH_AUTO.  Returns FQ_EINVAL on a bad q,
 * path or sizes, FQ_ENOMEM on host allocation failure, and FQ_ENOTSUP for a
 * plan beyond the kernels' 32-bit indices: 2^31 or more work items, tcgen05
 * tiles, or 128-byte rows in either arena.  No plan is made on an error. */
int fq_batched_plan_create(int q, int count, const int64_t *m, const int64_t *l, const int64_t *n,
                           fq_batch_plan **plan);
int fq_batched_plan_create_ex(int q, int count, const int64_t *m, const int64_t *l, const int64_t *n, int path,
                              fq_batch_plan **plan);

/* Bytes of device workspace the plan needs (64-byte aligned, caller-owned:
 * the work lists, and for tcgen05 products each group's two scratch buffers,
 * buffer b holding (m rounded up to 128 + n rounded up to 256) x (l rounded up
 * to 128) bytes for the largest of the group's products b, b + 2, ...), the
 * number of Four-Russians work items, of products on the tcgen05 path and of
 * their 128 x 256 tiles; -1 for a NULL plan. */
int64_t fq_batched_workspace_bytes(const fq_batch_plan *plan);
int64_t fq_batched_items(const fq_batch_plan *plan);
int64_t fq_batched_tc_products(const fq_batch_plan *plan);
int64_t fq_batched_tc_tiles(const fq_batch_plan *plan);

/* Copy the plan's work lists into `workspace` (synchronous on `stream`).  Once
 * per plan and workspace, before any fq_matmul_batched on them. */
int fq_batched_plan_upload(const fq_batch_plan *plan, void *workspace, void *stream);

/* All products of the plan (Section 2's method, or the exact tensor-core
 * contraction, per product).  A, B, C: DEVICE arrays of `count` device
 * pointers to planes buffers (A_p m x l, B_p l x n, C_p m x n; C_p must not
 * alias A_p or B_p); workspace: the uploaded workspace.  Enqueues, on
 * `stream`, for tcgen05 products one persistent kernel (conversion and
 * products), then for Four-Russians items one memset and one persistent
 * kernel; allocates nothing and never synchronises, so it may be captured in
 * a CUDA graph.  Launches sharing a workspace must not overlap on the GPU. */
int fq_matmul_batched(const fq_batch_plan *plan, const uint64_t *const *A, const uint64_t *const *B,
                      uint64_t *const *C, void *workspace, void *stream);

/* fq_matmul_batched in its launch stages, so that each can be timed on its
 * own: `stages` is a bit mask of
 *   FQ_BATCH_STAGE_TC    the persistent tcgen05 kernel of the tcgen05 products
 *                        (operand conversion and tiles, one launch),
 *   FQ_BATCH_STAGE_M4RM  the queue reset and the persistent Four-Russians kernel;
 * stages run in that order.  fq_matmul_batched is FQ_BATCH_STAGE_ALL.  Same
 * arguments and rules as fq_matmul_batched; FQ_EINVAL for a mask outside
 * 0 .. FQ_BATCH_STAGE_ALL. */
#define FQ_BATCH_STAGE_TC 1
#define FQ_BATCH_STAGE_M4RM 2
#define FQ_BATCH_STAGE_ALL 3
int fq_matmul_batched_stages(const fq_batch_plan *plan, const uint64_t *const *A, const uint64_t *const *B,
                             uint64_t *const *C, void *workspace, void *stream, int stages);

/* The path a plan gives product p: FQ_PATH_MMA (tcgen05) or FQ_PATH_M4RM;
 * -FQ_EINVAL for a NULL plan or p outside 0 .. count - 1.  Host only. */
int fq_batched_product_path(const fq_batch_plan *plan, int p);

/* Free a plan (NULL is fine). */
int fq_batched_plan_destroy(fq_batch_plan *plan);

/* Size of the fixed device array fq_matmul_batched_static works in. */
#define FQ_BATCH_STATIC_BYTES (1 << 20)

/* fq_matmul_batched for callers that cannot allocate device memory -- for
 * example code running inside a framework whose allocator owns all of the
 * GPU's memory, or a plug-in that must not call cudaMalloc because it would
 * synchronise the device under its host.  No workspace argument: the work list
 * and queue counter live in one FQ_BATCH_STATIC_BYTES array the library keeps
 * on every GPU that loads it (until the process exits), and no call allocates
 * or frees device memory.
 *   - A plan needing more than FQ_BATCH_STATIC_BYTES of workspace
 *     (fq_batched_workspace_bytes), or holding tcgen05 products (whose
 *     arenas do not fit; build it with FQ_PATH_M4RM), is refused with
 *     FQ_ENOTSUP.
 *   - Each call copies the plan's work list into the array on `stream` before
 *     its launch (the array keeps the previous call's contents otherwise).
 *   - All calls on a GPU share the one array: calls whose work overlaps on the
 *     GPU (for example on two streams) race and give wrong results.
 *   - Each call copies the work list from host memory, which a graph replay
 *     could not repeat: FQ_ENOTSUP while `stream` is being captured.  The
 *     copies are from pageable host memory, so a call must also not run
 *     while another thread captures a stream in cudaStreamCaptureModeGlobal
 *     (such a copy would invalidate that capture).
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current).  Under CUDA's lazy module
 *     loading that first use also loads the library's device code and the
 *     array on that device, which synchronises like an allocation: make the
 *     first call during set-up, before any timing-critical section.
 *   - The looked-up address (like the status word's) is kept for the life of
 *     the process: the library does not survive cudaDeviceReset.
 * The paper has no counterpart: this is an interface for allocation-free
 * callers, with the arguments and results of fq_matmul_batched. */
int fq_matmul_batched_static(const fq_batch_plan *plan, const uint64_t *const *A, const uint64_t *const *B,
                             uint64_t *const *C, void *stream);

/* ---- measured autotuning -----------------------------------------------------
 * fq_autotune times, on the caller's operands and stream (synchronously), the
 * M4RM planner's choice, every compiled M4RM kernel of field q and the
 * tensor-core path, and remembers the fastest for this exact (q, m, l, n):
 * later fq_matmul / fq_matmul_ex calls with FQ_PATH_AUTO, k = 0 and kernel = 0
 * on that shape use it.  C holds the product when it returns.  The cache is
 * process-wide host memory; fq_autotune_clear empties it.  q = 2, 3, 4, 5 or 7. */
typedef struct fq_tune_result {
  int path;           /* FQ_PATH_M4RM or FQ_PATH_MMA                        */
  int kernel;         /* 1-based compiled M4RM kernel, 0 = the M4RM planner   */
  float ms;           /* time of the chosen candidate                         */
  float ms_planner;   /* time of the M4RM planner's choice                    */
  float ms_mma;       /* time of the tensor-core path (0 if not run)          */
} fq_tune_result;

int fq_autotune(int q, int64_t m, int64_t l, int64_t n, const uint64_t *A, const uint64_t *B, uint64_t *C,
                void *stream, fq_tune_result *out);
/* The cache as a file, so that measurements survive the process:
 * fq_autotune_save writes every remembered choice to `path` as JSON,
 *   {"format": "fq-autotune-1", "entries": [[q, m, l, n, path, kernel], ...]};
 * fq_autotune_load merges such a file into the cache (its entries replace
 * remembered choices of the same shapes).  A file that is not exactly that
 * document, or holds an entry the library cannot honour (a field without
 * kernels, a negative size, a path other than FQ_PATH_M4RM / FQ_PATH_MMA, a
 * kernel outside the field's compiled ones, a tensor-core entry with a
 * kernel), is refused whole with FQ_EINVAL and nothing is merged; I/O
 * failures are FQ_EINVAL too, host allocation failures FQ_ENOMEM.  Host only. */
int fq_autotune_save(const char *path);
int fq_autotune_load(const char *path);
/* FQ_OK and the remembered choice for (q, m, l, n), or FQ_ENOTSUP if none. */
int fq_autotune_lookup(int q, int64_t m, int64_t l, int64_t n, int *path, int *kernel);
int fq_autotune_clear(void);

/* The path and kernel that fq_matmul_ex with FQ_PATH_AUTO, k = 0 and kernel = 0
 * takes for (q, m, l, n) on the current device: FQ_PATH_KARATSUBA for the
 * extension fields q = 8 .. 125, else the fq_autotune choice when one is
 * remembered, otherwise the path with the smaller modelled time (kernel 0, the
 * M4RM planner).  The model counts waves of one CTA per SM
 * times block steps times the measured cycles of one step of each path; it
 * picks the tensor-core path for small products (up to about 1024 on a side
 * for F_3), where the Four-Russians tables are not amortised over enough
 * rows.  Host-only apart from the device attribute query; FQ_EINVAL for a
 * bad q, a negative size or a null pointer, FQ_ECUDA if no device answers. */
int fq_auto_choice(int q, int64_t m, int64_t l, int64_t n, int *path, int *kernel);

/* Compiled M4RM kernels for field q (planner candidates).  fq_kernel_count
 * returns their number (0 for a bad q); fq_kernel_info describes kernel idx:
 * block size k, the most rows one CTA holds, columns per CTA and warps per CTA.
 * Host-only; returns FQ_EINVAL for a bad q or idx. */
int fq_kernel_count(int q);

/* The compiled M4RM kernel (1-based, as fq_options.kernel) that a direct
 * Four-Russians product of this shape runs with these options (opt may be
 * NULL): opt->kernel when set, else the fq_autotune choice when one is
 * remembered (AUTO path, k = 0), else the planner's.  Negative status on
 * error (-FQ_EINVAL for a bad q or shape, -FQ_ENOTSUP if no kernel has the
 * requested k).  Host-only apart from the device attribute query. */
int fq_planned_kernel(int q, int64_t m, int64_t l, int64_t n, const fq_options *opt);
int fq_kernel_info(int q, int idx, int *k, int *max_rows, int *cols, int *warps);

/* The library's scratch pool (one per device, created on first use) keeps the
 * memory it has handed out for later products instead of returning it at
 * every synchronisation.  fq_release_scratch synchronises the current device
 * and returns the pool's unused memory to the system.  Synchronous. */
int fq_release_scratch(void);

/* Wait for `stream`, then return and clear the first error kernels recorded on
 * the current device (FQ_EVALUE, FQ_ETIMEOUT), or FQ_OK.  Synchronous. */
int fq_status(void *stream);

/* Failure-path hooks, so that tests can drive the timeout path on purpose; no
 * product needs them.  Process-wide host settings read at each launch of the
 * Four-Russians kernels (a captured graph keeps the values of its capture).
 * Host only.
 *   fq_debug_wait_limit: later launches give up each bounded device wait (an
 *     mbarrier hand-over between the warps of a CTA, normally bounded at about
 *     two seconds) after `ns` nanoseconds of polling instead; ns <= 0 restores
 *     the default.  (A wait polls with mbarrier.try_wait, which may itself
 *     suspend the thread for a hardware-defined time, so a short wait can
 *     complete although it outlasts a very small limit.)
 *   fq_debug_stall_block: in later launches one thread of every CTA, on
 *     reaching k-row block `block`, also waits on a barrier that nothing ever
 *     completes -- a wait that always gives up; block < 0 turns it off.
 * A wait that gives up records FQ_ETIMEOUT for fq_status(); the CTA then stops
 * issuing copies, waits (with the default bound) for the copies it already
 * issued, skips the lookups whose tables it never received and exits: the
 * product is garbage but the device stays usable. */
int fq_debug_wait_limit(int64_t ns);
int fq_debug_stall_block(int64_t block);

/* Failure-path hook for host memory: after `after` further host allocation
 * points of batched-plan building (creation and fq_batched_plan_upload's host
 * image of the tables), the next one fails as an exhausted heap would, and
 * the call returns FQ_ENOMEM with no plan made and nothing enqueued; the hook
 * then disarms.  after < 0 disarms it.  Process-wide; host only; for tests. */
int fq_debug_fail_host_alloc(int64_t after);

/* Static text for a status code. */
const char *fq_error_string(int status);

/* Text of the last CUDA error seen by this library in the calling thread. */
const char *fq_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FQ_H */

/*
 * cwt.h -- C ABI of the GB300-native FFT-based continuous wavelet transform
 * (CWT) of multichannel EEG, after arXiv 2506.07793 (Nakanishi, "Novel
 * software for continuous wavelet analysis enable EEG real-time analysis on
 * portable computers").
 *
 * The method (Section "Fourier transformed formula", Eq. 2): for every
 * channel take one forward FFT of the zero-padded signal, multiply it by the
 * analytic Fourier-domain wavelet of each scale (Morlet, Eq. 3; Gabor, Eq. 4),
 * take one inverse FFT per (channel, scale) and reduce the result to complex
 * coefficients, power or phase (Section "Precision").  Padding follows Section
 * "Fast Fourier transform".  The wavelets are generated on the GPU once per
 * plan and reused (Section "Optimizing performance").
 *
 * Result definition.  For signal x[0..n) of channel c, padded length N and the
 * scale with carrier F_s (Hz) and sigma_s = n_cycles_s, the library returns
 *     coef[c][s][o] = sum_{m<n} x[m] * w_s[(d*o - m) mod N],  o < n_out,
 * where w_s is the N-periodised sampled Morlet wavelet normalised to unit
 * energy, d the decimation and n_out = ceil(n/d).  power = |coef|^2 and
 * phase = atan2(Im, Re) in (-pi, pi].  The GPU evaluates this with FFTs;
 * the values are those of the direct cyclic convolution, up to FP32 rounding.
 *
 * Conventions for every function below:
 *  - Every call returns a cwt_status and never throws or aborts across the ABI.
 *    Output arguments are written only when CWT_OK is returned.
 *  - "Device pointer" means memory of the plan's GPU (cudaMalloc, the torch
 *    caching allocator, or managed memory); "host pointer" means CPU memory
 *    (pinned memory makes the copies asynchronous-capable and faster).
 *  - Device buffers passed to cwt_execute must be 16-byte aligned; the caller
 *    owns them.  The plan owns its wavelet bank, tables and workspace.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device
 *    work is asynchronous on it; errors raised by kernels surface at the next
 *    call that synchronises (cwt_execute_host, cwt_plan_bank, profiling reads)
 *    or at the caller's own synchronisation.
 *  - A plan is not thread-safe, and its executions must not overlap on the
 *    GPU (they share the plan's spectrum workspace): issue them on one stream
 *    or synchronise in between.  Different plans are independent.
 *  - Layouts are row-major: signal [C][n]; every output [C][S][n_out].
 *    Complex outputs are interleaved (re, im) pairs of the I/O type.
 */
#ifndef CWT_GB300_CWT_H
#define CWT_GB300_CWT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cwt_plan_s *cwt_plan; /* opaque; created and freed by the library */

typedef enum {
    CWT_OK = 0,
    CWT_EINVAL = 1,        /* bad argument (value, pointer kind, alignment) */
    CWT_ENOMEM = 2,        /* device or host allocation failed */
    CWT_EUNSUPPORTED = 3,  /* valid request that this build does not implement */
    CWT_ECUDA = 4,         /* a CUDA runtime call failed (see cwt_plan_last_error) */
    CWT_EAGAIN = 5,        /* not enough data yet / nothing ready */
    CWT_EBUSY = 6,         /* admission refused: no slot or memory budget */
    /* 7 is not used: no kernel of this library waits on the device */
    CWT_EDEVICE = 8        /* a kernel reported an error: in the bounds-checked build
                              (-DCWT_BOUNDS_CHECK), an out-of-range shared-memory
                              access or index, named by cwt_plan_last_error */
} cwt_status;

typedef enum {
    CWT_WAVELET_MORLET = 0, /* Eq. 3 */
    CWT_WAVELET_GABOR = 1,  /* Eq. 4 (Morlet without the admissibility term) */
    CWT_WAVELET_GMW = 2     /* Eq. 5, generalized Morse wavelet with the Heaviside
                               step U(omega) in place of sign(omega); n_cycles[s]
                               holds beta_s and the options hold gamma */
} cwt_wavelet;

/* Output kinds, a bitmask (Section "Precision": real/imaginary, phase, power). */
enum { CWT_OUT_COMPLEX = 1u, CWT_OUT_POWER = 2u, CWT_OUT_PHASE = 4u };

typedef enum { CWT_PREC_FP32 = 0, CWT_PREC_TC_FP16 = 1, CWT_PREC_TC_BF16 = 2 } cwt_precision;
typedef enum { CWT_DTYPE_F32 = 0, CWT_DTYPE_F64 = 1 } cwt_dtype;

/* Padding policy (Section "Fast Fourier transform").  POW2 pads to the next
 * power of two (the choice the paper attributes to MNE-python), up to 131072.
 * SMOOTH is the paper's own policy: the smallest length >= max(samples, 32)
 * whose prime factors are 2, 3, 5 and 7.  Smooth lengths that are not powers
 * of two run on the mixed-radix kernels: one CTA per row where a radix
 * schedule of at most 32 values per thread and 512 threads covers N (every
 * smooth N <= 16384 but 15 in 14175 ... 16200), else a row of N = CL NL
 * points on a thread-block cluster of CL CTAs, with NL <= 16384 a scheduled
 * length and some such CL among 2 ... 8 (up to N = 131072; the split a plan
 * runs is cwt_smooth_cluster's, which may take up to 16 CTAs).
 * The 43 smooth lengths with neither (3^10 = 59049, 5^7 = 78125, and 41
 * from 84375 up, where every split leaves NL > 16384 or unscheduled) are
 * passed over: SMOOTH then gives the next one, and an explicit fft_length
 * of such a length is CWT_EUNSUPPORTED.
 * cwt_execute_batch does not take mixed-radix plans (CWT_EUNSUPPORTED). */
typedef enum { CWT_PAD_POW2 = 0, CWT_PAD_SMOOTH = 1 } cwt_pad_policy;

/* Edge handling (Section "Fourier transformed formula": the FFT path gives a
 * cyclic convolution, which approximates the simple convolution except near
 * the edges).  CYCLIC: the cyclic result over N = pad_policy(samples), the
 * paper's own computation.  LINEAR: the "same"-mode linear convolution of
 * the signal with the wavelet, by padding to N = pad_policy(samples + R + 1),
 * R the largest scale's support radius (cwt_support_radius: the envelope is
 * below 1e-9 of its peak beyond R samples), so that no wavelet wraps around;
 * the result then equals the linear convolution on [0, samples) up to that
 * envelope tail.  CWT_EUNSUPPORTED when samples + R + 1 exceeds 2^17. */
typedef enum { CWT_EDGE_CYCLIC = 0, CWT_EDGE_LINEAR = 1 } cwt_edge_mode;

/* Per-scale normalisation of the wavelet (Section "Precision" compares the
 * coefficients with MNE-python's, Table 1).  UNIT_ENERGY: the periodised
 * sampled wavelet has sum_m |w[m]|^2 = 1.  MNE: the convention MNE-python
 * documents for its Morlet wavelets (each wavelet divided by sqrt(0.5) times
 * its L2 norm), i.e. sum_m |w[m]|^2 = 2: every coefficient is sqrt(2) times
 * the unit-energy one and every power twice.  MNE also truncates each
 * wavelet at 5 sigma_t (an envelope below 4e-6 of its peak); the library
 * keeps the untruncated wavelet, so coefficients differ from MNE's by that
 * tail (a comparison with MNE itself is not made here: MNE is not part of
 * this library's dependencies). */
typedef enum { CWT_NORM_UNIT_ENERGY = 0, CWT_NORM_MNE = 1 } cwt_normalization;

/* Kernel identifiers for the profiling counters. */
typedef enum {
    CWT_KERNEL_BANK = 0,        /* wavelet-bank + band generation (plan creation) */
    CWT_KERNEL_FORWARD_FFT = 1, /* per-channel forward FFT */
    CWT_KERNEL_SCALE_BLOCK = 2, /* fused multiply + inverse FFT + reduce + store */
    CWT_KERNEL_BATCH = 3,       /* persistent batch kernel (one graph launch) */
    CWT_KERNEL_COUNT = 4
} cwt_kernel_id;

/* One epoch of a batch (cwt_execute_batch).  Offsets are in elements of the
 * packed arrays: the epoch's signal is the [C][samples] block starting at
 * in_offset, and its outputs are the [C][S][ceil(samples/d)] blocks starting
 * at out_offset in each requested output array (complex arrays count complex
 * elements). */
typedef struct {
    long long in_offset;
    long long out_offset;
    int samples;  /* 1 <= samples <= the plan's samples and <= 8192 */
    int reserved;
} cwt_epoch;

/* What the batch path did last (cwt_plan_batch_stats). */
typedef struct {
    int items;              /* work items (epoch, channel group) of the last batch */
    int grid;               /* persistent CTAs launched */
    int inverse_radix;      /* autotuned points per thread of the inverse FFTs (16 or 32) */
    int order;              /* autotuned item order: 0 largest FFT first, 1 input order */
    int tuned;              /* 1 once the autotuner has chosen for this batch shape */
    int reserved;
    double tune_ms[4];      /* candidate times: (16,0), (32,0), (16,1), (32,1); -1 for a
                               radix-16 candidate the batch rules out (an inverse row
                               longer than 4096 points, at N_e = 8192 and odd d) */
    long long graph_launches;
    size_t bank_bytes;      /* device bytes of the per-length wavelet banks */
} cwt_batch_stats;

typedef struct {
    int precision;  /* cwt_precision of the inverse FFTs (default FP32).  TC_FP16 and
                       TC_BF16 run their radix-16 stages as DFT matrix products on
                       the tensor cores with hi/lo split operands and FP32
                       accumulation (the Cooley-Tukey factorisation of Section
                       "Fast Fourier transform"; error within 2e-3 of the row's
                       peak power): power-of-two N of 16384 ... 131072 only (else
                       CWT_EUNSUPPORTED); not for cwt_execute_batch */
    int decimation; /* keep every d-th output sample, d >= 1 (default 1) */
    int pad_policy; /* cwt_pad_policy (default CWT_PAD_POW2) */
    int fft_length; /* 0: from pad_policy; else an explicit N >= samples that is a
                       power of two the build supports or a 2,3,5,7-smooth
                       length the mixed-radix kernels run (see cwt_pad_policy) */
    int io_dtype;   /* cwt_dtype of the signal and of every output (default F32);
                       F64 is converted to FP32 on load and back on store */
    int edge_mode;  /* cwt_edge_mode (default CWT_EDGE_CYCLIC) */
    double gmw_gamma; /* gamma of the generalized Morse wavelet (Eq. 5), > 0,
                         default 3; read only for CWT_WAVELET_GMW */
    int normalization; /* cwt_normalization of each scale's wavelet (default
                          CWT_NORM_UNIT_ENERGY) */
    int specialize;    /* 1: for a smooth N (not a power of two) with no
                          fixed-length kernel compiled in, compile the fixed-length
                          kernels for N's schedule -- or for the local length of
                          its cluster split -- at plan creation (NVRTC, about a
                          second, cached per process; Section "Fast Fourier
                          transform");
                          if that fails the plan runs the runtime-schedule kernels
                          (cwt_plan_info.specialized, cwt_plan_last_error).
                          2: for a smooth N, compile up to eight candidate
                          schedules of N -- or of its cluster split's local
                          length -- (the scheduler's, its passes on two other
                          thread counts, then the cost model's two cheapest
                          radix sets in each pass order) and keep the
                          fastest on the plan's own rows, the compiled-in
                          kernel competing where there is one (a few seconds;
                          cwt_plan_info.radices reports the winner).
                          0 (default): never compile at plan creation.
                          Compiled modules are kept per process; with the
                          environment variable CWT_JIT_CACHE_DIR naming a
                          writable directory, also on disk, and later processes
                          load them instead of compiling */
    int reserved[6];
} cwt_options;

typedef struct {
    int channels, samples, scales;
    int fft_length;     /* N */
    int n_out;          /* ceil(samples / decimation) */
    int decimation;
    int fold;           /* spectral fold factor f (power of two dividing d) */
    int inverse_length; /* N / fold: size of each inverse FFT */
    int device;         /* CUDA ordinal the plan lives on */
    int io_dtype;
    unsigned output_kinds;
    size_t workspace_bytes; /* device bytes owned by the plan */
    double bank_ms;         /* GPU time of the bank generation at creation */
    int radices[8];         /* smooth N: the inverse FFT's radix schedule, 0-terminated
                               (all 0 for powers of two) */
    int inlined_pair[2];    /* smooth N: the radix pair of the inlined kernel that runs
                               it, or 0, 0 for the generic mixed-radix kernel */
    int fixed_kernel;       /* smooth N: 1 when the scale-block kernel runs from a build
                               compiled for exactly this N and radix schedule (27
                               whole-second EEG lengths from 500 to 15000, e.g. 10000,
                               12000, 7500, 3000, 1250; on a cluster, a local
                               length of 15360, 15000 or 10000, e.g. N = 122880,
                               60000, 20000),
                               else 0; the forward FFTs then run on the same schedule */
    int precision;          /* cwt_precision of the inverse FFTs */
    int cluster;            /* CTAs that share each inverse FFT (a thread-block cluster
                               over distributed shared memory): 1 when one CTA holds the
                               row (at most 16384 points), else 2 ... 16, each CTA holding
                               inverse_length / cluster points (powers of two: 2, 4, 8;
                               smooth lengths: cwt_smooth_cluster's split); radices then
                               describe those points' passes */
    int specialized;        /* 1 when the plan runs kernels compiled at its creation
                               (cwt_options.specialize), 2 when they were chosen among
                               candidate schedules by timing (specialize = 2) */
} cwt_plan_info_t;

/* Human-readable name of a status.  Never NULL. */
const char *cwt_status_str(cwt_status s);

/* Fill *opt with defaults: FP32, d = 1, CWT_PAD_POW2, N from the policy, F32
 * I/O, CWT_EDGE_CYCLIC, gmw_gamma 3, CWT_NORM_UNIT_ENERGY. */
cwt_status cwt_options_init(cwt_options *opt);

/* Padded FFT length N for `samples` under `pad_policy` (Section "Fast Fourier
 * transform"): POW2, the next power of two >= max(samples, 32); SMOOTH, the
 * smallest 2,3,5,7-smooth length >= max(samples, 32) that the mixed-radix
 * kernels run (see cwt_pad_policy).  Writes *n_fft.  CWT_EINVAL if samples < 1
 * or the policy is unknown; CWT_EUNSUPPORTED if N exceeds the largest
 * supported length, 2^17 under both policies (lengths above 2^14 run each row
 * on a thread-block cluster).  Host-only; no CUDA call. */
cwt_status cwt_fft_length(int samples, int pad_policy, int *n_fft);

/* Support radius of one scale's wavelet at sampling rate fs, in samples: the
 * envelope |psi(t)| stays below 1e-9 of its peak for |t| > radius / fs (the
 * padding of CWT_EDGE_LINEAR).  Morlet and Gabor (Eq. 3, Eq. 4): their
 * Gaussian envelope, ceil(6.5 a fs), a = n_cycles / (2 pi freq_hz).  GMW
 * (Eq. 5; n_cycles holds beta, gmw_gamma its gamma): measured from the
 * spectrum by an FP64 inverse FFT on the host (it scales as 1 / freq_hz).
 * Writes *radius.  CWT_EINVAL for arguments cwt_plan_create would refuse;
 * CWT_EUNSUPPORTED when the radius exceeds 2^17 samples.  Host-only; no CUDA
 * call. */
cwt_status cwt_support_radius(int wavelet, double freq_hz, double n_cycles, double gmw_gamma, double fs,
                              int *radius);

/* The schedule the mixed-radix kernels run for a 2,3,5,7-smooth length n_fft
 * that is not a power of two (Section "Fast Fourier transform"), as
 * cwt_plan_info reports it for a plan of that length: radices[8] the inverse
 * FFT's passes in order, 0-terminated; *threads the threads per row;
 * inlined_pair[2] the radix pair of the inlined kernel, or 0, 0 for the
 * generic one; *fixed_kernel 1 when the scale block runs from a kernel
 * compiled for exactly this length and schedule.  Outputs are host memory
 * owned by the caller.  CWT_EINVAL for a NULL output; CWT_EUNSUPPORTED when
 * n_fft is a power of two, not 2,3,5,7-smooth, outside [32, 16384] or one of
 * the lengths no schedule covers (see cwt_pad_policy).  Host-only; no CUDA
 * call. */
cwt_status cwt_smooth_schedule(int n_fft, int *radices, int *threads, int *inlined_pair,
                               int *fixed_kernel);

/* The row layout a plan of the 2,3,5,7-smooth length n_fft (not a power of
 * two, 32 ... 131072) runs with cwt_options.specialize = specialize (Section
 * "Fast Fourier transform"), as cwt_plan_info reports it before any
 * plan-time tuning: *cluster 1 for one CTA per row, else the CTAs of the
 * cluster split N = cluster x NL; radices[8] the passes of N's (of NL's)
 * schedule, 0-terminated; *fixed_kernel 1 when that schedule is compiled in
 * for this cluster size.  The split prefers local rows two CTAs per SM hold
 * on kernels built for that: fewest passes, then the smallest cluster; sizes
 * above 8 CTAs (non-portable clusters) only on compiled-in local rows or,
 * with specialize != 0, on kernels compiled at plan creation (such a
 * cluster needs a GPU partition whose GPCs hold it -- a whole GB300 does;
 * elsewhere its launch fails with CWT_ECUDA).  Outputs are
 * host memory owned by the caller.  CWT_EINVAL for a NULL output or
 * specialize outside 0 ... 2; CWT_EUNSUPPORTED for a length no kernel runs.
 * Host-only; no CUDA call. */
cwt_status cwt_smooth_cluster(int n_fft, int specialize, int *cluster, int *radices, int *fixed_kernel);

/* The plan-time compile of cwt_options.specialize for a smooth n_fft that is
 * not a power of two -- its one-CTA schedule, or its cluster split N = CL NL
 * (see cwt_pad_policy) -- for sm_103a, without a device (a check that the
 * embedded kernel source compiles): CWT_OK, CWT_EUNSUPPORTED when n_fft is
 * not such a length, or CWT_ECUDA when the compiler fails; the compiler's log
 * goes to `log` (host memory of log_len bytes, may be NULL), NUL-terminated.
 * Host-only; no CUDA runtime call. */
cwt_status cwt_specialize_check(int n_fft, char *log, size_t log_len);

/*
 * cwt_plan_create -- validate, pick N, allocate the plan's device memory on
 * the current CUDA device and generate the wavelet bank there in FP64
 * (Eq. 3/4/5 summed over aliases, normalised to unit energy, rounded to
 * FP32) together with each scale's non-negligible band (Section "Optimizing
 * performance": wavelets are generated in GPU memory first).
 *   channels, samples  C >= 1, n >= 1
 *   fs                 sampling rate in Hz, > 0
 *   freqs_hz[n_freqs]  host array, each 0 < F < fs/2 (Morlet/Gabor: the
 *                      carrier; GMW: the peak frequency of the spectrum)
 *   n_cycles[n_freqs]  host array, each > 0 (Morlet/Gabor: sigma of Eq. 3;
 *                      GMW: beta of Eq. 5, at most 1000)
 *   wavelet            cwt_wavelet
 *   output_kinds       non-empty subset of CWT_OUT_*
 *   opt                NULL for defaults
 * On CWT_OK *out holds a new plan (free with cwt_plan_destroy).  Argument
 * errors are reported before any CUDA call.  Blocks until the bank is built.
 * A scale that the N-point grid cannot represent is CWT_EINVAL: one whose
 * alias-summed spectrum is below 1e-150 on every DFT bin, so that its
 * unit-energy normalisation would underflow in FP64 (a carrier far below
 * the first bin, e.g. 1.5 Hz with 7 cycles in a 32-point window at 500 Hz,
 * where the first bin lies at ten times the carrier).  Scales below the
 * first bins but above that floor are computed exactly like the others.
 */
cwt_status cwt_plan_create(cwt_plan *out, int channels, int samples, double fs,
                           const double *freqs_hz, int n_freqs, const double *n_cycles,
                           int wavelet, unsigned output_kinds, const cwt_options *opt);

/* Free the plan and its device memory (synchronises the device work of the
 * plan first).  NULL is accepted. */
cwt_status cwt_plan_destroy(cwt_plan plan);

/* Describe the plan (host-only, no synchronisation). */
cwt_status cwt_plan_info(cwt_plan plan, cwt_plan_info_t *info);

/* Device bytes owned by the plan (0 for NULL). */
size_t cwt_plan_workspace_bytes(cwt_plan plan);

/* Text of the last CUDA error the plan saw ("" if none).  Never NULL. */
const char *cwt_plan_last_error(cwt_plan plan);

/*
 * cwt_execute -- the hot path (Eq. 2): forward FFT of every channel, then one
 * fused kernel per scale block that multiplies by the wavelet spectrum,
 * inverse-FFTs on chip, reduces and stores only the requested outputs.
 *   d_signal  device [C][n] of io_dtype
 *   d_complex device [C][S][n_out] complex (2 x io_dtype), or NULL
 *   d_power   device [C][S][n_out] io_dtype, or NULL
 *   d_phase   device [C][S][n_out] io_dtype, or NULL
 * Exactly the kinds given at plan creation must be non-NULL.  Pointers must
 * be device memory of the plan's GPU and 16-byte aligned (else CWT_EINVAL).
 * Asynchronous on `stream`.
 */
cwt_status cwt_execute(cwt_plan plan, const void *d_signal, void *d_complex, void *d_power,
                       void *d_phase, void *stream);

/*
 * cwt_execute_host -- the same transform with HOST buffers: copies the signal
 * to the plan's device staging buffer, runs cwt_execute on `stream` and waits
 * for the outputs.  An output buffer in page-locked host memory that the
 * device can address (cudaHostAlloc / cudaMallocHost, cudaHostRegister with
 * mapping, e.g. torch pin_memory(); 16-byte aligned) is written directly by
 * the kernels' epilogues over the host link, with no staging copy; any other
 * output goes to a device staging buffer and is copied back.  Staging buffers
 * are allocated on the first call and kept by the plan.  Same layouts as
 * cwt_execute.  Returns when the outputs are in host memory.
 */
cwt_status cwt_execute_host(cwt_plan plan, const void *h_signal, void *h_complex, void *h_power,
                            void *h_phase, void *stream);

/*
 * cwt_execute_batch -- many epochs of uneven length in one persistent launch
 * replayed from a CUDA graph.  Epoch e is the same transform as cwt_execute
 * on its own samples (padded length N_e = next power of two >= max(n_e, 32),
 * or >= n_e + R + 1 with CWT_EDGE_LINEAR,
 * Section "Fast Fourier transform"), with the plan's channels, scales,
 * decimation and output kinds.  The paper loops over recordings in Python
 * (Section "Wavelength and flexibility"); here they share one launch.
 *   epochs[n_epochs]  host array of cwt_epoch (offsets in elements)
 *   d_in              device packed float32 input
 *   d_complex / d_power / d_phase  device packed outputs (exactly the plan's kinds)
 * Requires an F32 plan.  The first batch of a new shape generates the banks
 * for its lengths (allocating and waiting) and runs the autotuner, which times
 * four schedules on this batch and keeps the fastest; later batches of the
 * same shape only replay the graph.  Asynchronous on `stream` otherwise.
 * CWT_EUNSUPPORTED for F64 plans, smooth-padded plans, or epochs whose
 * padded length would exceed 8192 samples.  CWT_EINVAL (before any device
 * work) when an epoch's N_e cannot represent one of the plan's scales (the
 * 1e-150 floor of cwt_plan_create).
 */
cwt_status cwt_execute_batch(cwt_plan plan, const cwt_epoch *epochs, int n_epochs, const void *d_in,
                             void *d_complex, void *d_power, void *d_phase, void *stream);

/* Statistics of the plan's batch path (zeros before the first batch). */
cwt_status cwt_plan_batch_stats(cwt_plan plan, cwt_batch_stats *stats);

/* ---------------------------------------------------------------------------
 * Streaming (live EEG).  The paper's aim is real-time analysis (Abstract;
 * Discussion: 64-channel EEG transformed several times per second).  A server
 * keeps many live streams; each hop of H = ceil(fs * hop_seconds) new samples
 * yields the CWT power of the window x[e - W, e) (cyclic, Eq. 2 with N = W,
 * zeros before the first sample) at the H window positions
 * [W - D - H, W - D), D = floor((W - H) / 2), i.e. absolute sample times
 * [e - D - H, e - D).  Every ready hop of every open stream goes into the
 * next cwt_server_step launch (continuous batching).
 * ------------------------------------------------------------------------- */
typedef struct cwt_server_s *cwt_server;

typedef struct {
    int max_streams;          /* stream slots (default 32) */
    int window;               /* W = N; only 2048 is built */
    double hop_seconds;       /* hop length in seconds (default 0.05) */
    size_t mem_budget_bytes;  /* device bytes for streams (0 = no limit) */
    unsigned output_kinds;    /* only CWT_OUT_POWER is built */
    int reserved0;
    double gmw_gamma;         /* gamma for CWT_WAVELET_GMW (default 3) */
    int reserved[4];
} cwt_server_options;

typedef struct {
    int open_streams;
    int reserved;
    long long admitted, refused;  /* cwt_stream_open outcomes since the last reset */
    long long hops, launches;     /* hops completed, batched launches */
    long long coefficients;       /* power values delivered (C * S * H per hop) */
    size_t device_bytes;          /* device memory held by banks and streams */
    double latency_p50_s, latency_p99_s, latency_max_s, latency_mean_s;
    double span_s;                /* first hop ready -> last hop done */
} cwt_server_stats_t;

cwt_status cwt_server_options_init(cwt_server_options *opt);

/* A server for the scales freqs_hz/n_cycles (host arrays, as cwt_plan_create)
 * on the current device.  Streams are opened later with their own fs. */
cwt_status cwt_server_create(cwt_server *out, const double *freqs_hz, const double *n_cycles,
                             int n_freqs, int wavelet, const cwt_server_options *opt);
/* Waits for in-flight work, frees everything. */
cwt_status cwt_server_destroy(cwt_server srv);

/* Admit a stream of `channels` channels sampled at fs Hz (every frequency must
 * be < fs/2 and representable on the window's W-point grid at fs, as in
 * cwt_plan_create; else CWT_EINVAL).  CWT_EBUSY when no slot is free or its
 * device memory would exceed the budget (the refusal is counted).  Generates
 * the bank for a new fs and grows the server's batch buffers to hold
 * kMaxPending (8) hops of every open stream, waiting for the batches in
 * flight if it has to replace them.  Call cwt_stream_open, cwt_server_step
 * and cwt_stream_close from one thread. */
cwt_status cwt_stream_open(cwt_server srv, int channels, double fs, int *stream_id);

/* Append k new samples per channel: samples is [channels][k] float32, host or
 * device memory.  Hops completed by these samples become ready.  CWT_EBUSY
 * (nothing is pushed) if k > 8 * H or if the stream would then hold more than
 * 8 hops not yet pulled: step the server and pull first.  One thread feeds a
 * given stream. */
cwt_status cwt_stream_push(cwt_server srv, int stream_id, const float *samples, int k);

/* Launch one batch with every ready hop of every open stream, asynchronously
 * on the server's own CUDA stream (two batches may be in flight; a third call
 * waits for the oldest).  *hops_launched (may be NULL) receives the count.
 * Allocates nothing: the batch buffers were sized when the streams were
 * admitted.  Pushes copy on a separate CUDA stream, and the batch waits only
 * for the pushes issued before this call. */
cwt_status cwt_server_step(cwt_server srv, int *hops_launched);

/* Wait until every launched batch has completed. */
cwt_status cwt_server_sync(cwt_server srv);

/* Copy up to max_hops completed hops, oldest first, into out: each hop is a
 * [channels][S][H] float32 block (power).  *first_sample receives the absolute
 * time (in samples) of the first returned output (may be NULL).  CWT_EAGAIN
 * with *n_hops = 0 when none is complete yet. */
cwt_status cwt_stream_pull(cwt_server srv, int stream_id, float *out, int max_hops, int *n_hops,
                           long long *first_sample);

/* Close a stream (waits for its launched hops, frees its slot and memory). */
cwt_status cwt_stream_close(cwt_server srv, int stream_id);

/* Latency percentiles (ready -> output in host memory), throughput counters. */
cwt_status cwt_server_stats(cwt_server srv, cwt_server_stats_t *stats);
cwt_status cwt_server_reset_stats(cwt_server srv);

/*
 * cwt_plan_bank -- copy the plan's wavelet bank to host memory (synchronous).
 *   h_bank        [S][N] float32: the real spectrum W_s[k] / N actually used
 *                 (the 1/N of the inverse FFT is folded in), or NULL
 *   h_band_start  [S] first bin of each scale's band (0..N-1), or NULL
 *   h_band_len    [S] number of bins in the band (the band wraps mod N), or NULL
 * Bins outside the band hold values below 1e-10 of the scale's peak and are
 * skipped by the kernels.
 */
cwt_status cwt_plan_bank(cwt_plan plan, float *h_bank, int *h_band_start, int *h_band_len);

/*
 * cwt_fft -- batched, unnormalised complex FFT with the library's Stockham
 * kernels (a building block, exposed for testing and reuse).
 *   d_in, d_out  device [batch][n] complex64, 16-byte aligned; may alias
 *   n            power of two, 32 <= n <= 131072 (above 16384: one cluster per row)
 *   direction    -1: sum x[m] e^{-2 pi i k m / n};  +1: e^{+2 pi i ...}
 * Asynchronous on `stream`.
 */
cwt_status cwt_fft(const void *d_in, void *d_out, int n, int batch, int direction, void *stream);

/*
 * Profiling (Section "Comparison between devices and software" times each
 * method; here each kernel is timed with CUDA events on its own stream).
 * cwt_plan_set_profiling(plan, 1) makes every later launch of the plan record
 * an event pair on its stream; cwt_plan_profile_read waits for the recorded
 * events of `kernel` (a cwt_kernel_id), returns their count and summed
 * milliseconds, and with reset != 0 forgets them.
 */
cwt_status cwt_plan_set_profiling(cwt_plan plan, int enable);
cwt_status cwt_plan_profile_read(cwt_plan plan, int kernel, int *launches, double *total_ms,
                                 int reset);

/*
 * cwt_measure_peak -- measured compute peak of the current GPU in TFLOP/s,
 * the denominator of the benchmark's compute-side roofline fractions (the
 * paper has no counterpart; a measurement aid).  what = 0: FP32 FMA
 * throughput (8 independent fma.rn.f32 chains per thread, 8 CTAs of 256
 * threads per SM, 2 flops per FMA); 1: mma.sync.m16n8k16 with FP16 operands
 * and FP32 accumulation (4 independent accumulators per warp, 4096 flops per
 * MMA), the instruction of the tensor-core inverse FFTs; 2: the same with
 * BF16.  One warm-up and one timed launch of a few tens of milliseconds,
 * CUDA events on the legacy default stream; synchronous.  CWT_EINVAL for an
 * unknown `what` or NULL `tflops`.
 */
cwt_status cwt_measure_peak(int what, double *tflops);

/*
 * cwt_execute_noalloc -- the Morlet transform of cwt_plan_create +
 * cwt_execute (power-of-two padding, no decimation, float32 signal and
 * outputs) for callers that must not allocate GPU memory while they run: a
 * real-time EEG / BCI processing loop, where a cudaMalloc or cudaFree can
 * synchronise the device and blow the loop's deadline, or a plug-in whose host
 * application owns the GPU memory budget.  The paper has no counterpart; it is
 * an addition of this library.
 *
 * It allocates nothing.  The caller passes the signal and the outputs; the
 * twiddle table, wavelet bank, band table and spectra live in one fixed
 * device array of CWT_NOALLOC_SCRATCH_BYTES that every GPU loading this
 * library holds until the process exits.  The bank is regenerated (FP64, as
 * in cwt_plan_create) on every call, so no plan is needed.
 *   d_signal   device [channels][samples] float32, 16-byte aligned
 *   fs, freqs_hz[n_freqs], n_cycles[n_freqs]  as for cwt_plan_create (host arrays)
 *   d_complex  device [channels][n_freqs][samples] complex64, or NULL
 *   d_power, d_phase  device [channels][n_freqs][samples] float32, or NULL
 *              (at least one output non-NULL; all 16-byte aligned)
 * Size limit: with N = cwt_fft_length(samples), S = n_freqs, C = channels
 * and r(x) = x rounded up to a multiple of 256 bytes, the request must satisfy
 *   1 MiB + r(16 S) + r(8 S ceil(N/256)) + r(8 S) + r(4 S N) + 8 C N
 *       <= CWT_NOALLOC_SCRATCH_BYTES
 * (each region of the array starts on a 256-byte boundary), e.g. 64 channels
 * x 10000 samples x 100 scales fits; larger requests return CWT_EINVAL
 * before any device work.
 * The first call on a device (the current device) resolves the array's device
 * address and writes its twiddle table, then waits for that on `stream`.  No
 * call may be made inside a stream capture: each one copies freqs_hz and
 * n_cycles from pageable host memory (cudaMemcpyAsync), which a captured
 * stream refuses or would replay from host memory the caller may have freed.
 * The address is kept for the
 * life of the process: do not call this entry point again on a device after
 * cudaDeviceReset.  Every call copies freqs_hz and n_cycles into the array
 * (so the caller may reuse them as soon as the call returns), reuses the same
 * array and overwrites everything it reads, so nothing needs clearing between
 * calls; calls that overlap on the GPU (unordered streams, other host
 * threads) race on it and must be serialised by the caller.  Its kernels run
 * on `stream`; the call returns without waiting for them (except the first
 * call's set-up).
 */
#define CWT_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
cwt_status cwt_execute_noalloc(const float *d_signal, int channels, int samples, double fs,
                               const double *freqs_hz, const double *n_cycles, int n_freqs,
                               void *d_complex, float *d_power, float *d_phase, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CWT_GB300_CWT_H */

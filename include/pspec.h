/*
 * pspec.h — C ABI of libpspec, the GB300 (sm_103a) implementation of the
 * spherical-harmonic FFT estimator of power-spectrum multipoles P_l(k) with a
 * moving (local plane-parallel) line of sight, and of the P(k, mu) wedges built
 * from them (Hand, Li, Slepian & Seljak 2017, arXiv:1704.02357).
 *
 * Operations and where the paper defines them
 *   pspec_paint       Sec. 2.1 eq. FKP-density (F = w [n - alpha n_s], I, alpha) and
 *                     the shot-noise term after eq. Pell-full; Sec. 2.3 mass assignment
 *                     (CIC / TSC) and the interlaced second mesh.
 *   pspec_multipoles  Sec. 2.1 eqs. Pell-ours and Fell with the real harmonics of
 *                     eq. real-Ylm (2l+1 real-to-complex transforms per multipole);
 *                     Sec. 2.3 interlacing, window compensation and the inverse
 *                     transform before the Y_lm weighting; k-shell averages.
 *   pspec_wedges      Sec. 2.2 eqs. wedge-est and Lbar.
 *
 * Conventions (shared by every entry point)
 *   - Mesh: N^3 nodes at corner + i*H, H = box_size/N, index order (x, y, z), z fastest.
 *   - Forward transforms use exp(-i k.x); integer frequencies n in [-N/2, N/2).
 *   - alpha = sum of data completeness weights / sum of randoms completeness weights;
 *     I = alpha * sum_randoms nbar w_c w_fkp^2; S = sum_data v^2 + alpha^2 sum_randoms v^2,
 *     v = w_c * w_fkp, w_fkp = 1/(1 + nbar P0) (1 when P0 = 0). S is subtracted from
 *     l = 0 only.
 *   - When interlacing or compensation is on, modes with some n_d = -N/2 are zeroed
 *     before the inverse transform. Modes with some n_d = -N/2, and k = 0, are never
 *     binned. Mode n lies in bin b iff t_b <= |n|^2 < t_{b+1}, t_b = (k_b L / 2pi)^2 (FP64).
 *
 * Ownership and errors
 *   - Every call returns a pspec_status. No exception crosses the ABI. pspec_strerror()
 *     names a status; pspec_last_error() gives the detail of the last failure on a context.
 *   - The caller owns every pointer it passes. Device memory for meshes, spectra and
 *     tables is one caller-provided workspace (size from pspec_workspace_size) that must
 *     stay allocated until pspec_destroy; the library allocates no device memory itself.
 *   - All device work is enqueued on the stream given to pspec_create, in call order.
 *     Calls on one context are not thread-safe; distinct contexts are independent.
 *   - Host output pointers are written before the call returns (the call synchronises
 *     the stream). The *_device variants write device buffers and return without
 *     synchronising.
 *   - Invalid arguments give PSPEC_EINVAL and leave the context usable. A CUDA error
 *     gives PSPEC_ECUDA; the context should then be destroyed.
 */
#ifndef PSPEC_H
#define PSPEC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t pspec_status;
enum {
  PSPEC_OK = 0,
  PSPEC_EINVAL = 1,        /* bad argument: sizes, edges, l, pointers, non-finite inputs */
  PSPEC_ENOMEM = 2,        /* workspace too small */
  PSPEC_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
  PSPEC_ETIMEOUT = 4,      /* a bounded device-side wait ran out */
  PSPEC_ECANCELED = 5,     /* the caller cancelled the work */
  PSPEC_EUNSUPPORTED = 6,  /* valid but not implemented here: odd l, l > 16, N not 2^a or 3*2^a */
  PSPEC_ESTATE = 7         /* call out of order (e.g. multipoles before paint) */
};

enum { PSPEC_WINDOW_CIC = 2, PSPEC_WINDOW_TSC = 3 };   /* value = order p of sinc^p */
/* PSPEC_FP32: FP32 meshes and transforms with FP64 sums and bins; the harmonic transforms and the
 * inverse transform add exactly (each value a float on a power-of-two grid plus a float
 * remainder) and round once per shared-memory exchange and pass, which keeps the multipoles
 * within 1e-5 (l <= 4) / 1e-4 (l <= 16) of an FP64 evaluation at 512^3.
 * PSPEC_FP32_PLAIN: every transform a plain FP32 radix tree (faster; rounds at every add level).
 * PSPEC_FP64: FP64 throughout. */
enum { PSPEC_FP32 = 0, PSPEC_FP64 = 1, PSPEC_FP32_PLAIN = 2 };
enum { PSPEC_POS_F64 = 0, PSPEC_POS_F32 = 1 };
#define PSPEC_MAX_ELL 16
#define PSPEC_MAX_KBINS 4096
#define PSPEC_MAX_MU 64

typedef struct {
  int32_t nmesh;           /* N: even, 8 <= N <= 1024, N = 2^a or 3*2^a */
  int32_t window;          /* PSPEC_WINDOW_CIC or PSPEC_WINDOW_TSC */
  int32_t interlaced;      /* 0/1: paint a second mesh shifted by H/2 (Sec. 2.3) */
  int32_t compensate;      /* 0: none; 1: divide by prod_d sinc^p(pi n_d/N); 2: divide by
                              prod_d sqrt(C_p(n_d)), C_p the alias sum of sinc^{2p} in the
                              closed form of Jing (2005) (removes the aliased shot noise of a
                              non-interlaced mesh on average); 3: leave the field uncompensated
                              and divide each mode's binned product by prod_d sinc^{2p} (no
                              inverse transform without interlacing) */
  int32_t precision;       /* PSPEC_FP32, PSPEC_FP32_PLAIN or PSPEC_FP64 (see above) */
  int32_t ell_max;         /* largest l this context will be asked for, 0..16 */
  double box_size;         /* L */
  double box_corner[3];    /* position of node (0,0,0) */
  double observer[3];      /* origin of the line of sight */
  double P0;               /* FKP P0; 0 gives w_fkp = 1 */
  double nbar;             /* n̄ used for particles whose catalog has no nbar array */
  int64_t max_group_bytes; /* cap on the per-group spectrum buffers; 0 = one whole multipole */
  int64_t max_particles;   /* data + randoms the tile-binned paint is sized for (FP32 meshes;
                              148 bytes of workspace per particle). That paint sums each cell
                              exactly (64-bit fixed point) and rounds it once, so the meshes do
                              not depend on the order of the additions. 0, a larger catalog pair
                              or FP64 meshes use direct atomic painting (FP32 meshes: atomics in
                              FP32, whose rounding depends on the order of the additions) */
  int32_t cache_randoms;   /* 0/1: reserve meshes for pspec_set_randoms / pspec_run_batch */
  int32_t ylm_table;       /* FP32 contexts, l_max >= 2: 0 = hold Y_lm(khat) of every stored mode
                              for l = 2..l_max, evaluated in FP64 at creation and rounded once
                              to FP32 (4 bytes per mode and harmonic: 41 GB at 512^3, l_max = 16),
                              when that takes at most PSPEC_YLM_TABLE_AUTO_MAX bytes; -1 = never.
                              Without the table the binning pass evaluates Y_lm(khat) in FP32;
                              its rounding is biased by a few percent of an ulp over a k shell,
                              which lets ~4e-9 of the shot-noise power into P_l (l >= 2) */
  int32_t cartesian;       /* 0/1 (FP32 contexts): also hold the k-space factors of the Cartesian
                              decomposition (21 values per stored mode, FP64-built, 5.6 GB at
                              512^3) for pspec_multipoles_cartesian */
} pspec_params;
#define PSPEC_YLM_TABLE_AUTO_MAX ((int64_t)64 << 30)
/* With ylm_table = 0, FP32 contexts also hold Y_lm(rhat) of every mesh node for l = 2..l_max
 * (even l), evaluated in FP64 at creation and rounded once to FP32 (4 bytes per node and
 * harmonic: 7.5 GB at 512^3, l_max = 4; 82 GB at l_max = 16), when that takes at most
 * PSPEC_YLM_RTABLE_AUTO_MAX bytes. The Y-weighted transforms read their weights from it;
 * without it they evaluate Y_lm(rhat) in FP32, whose errors are coherent over the sphere and
 * leak ~1e-4 of P_14 (and ~2e-5 of a small P_4) at 512^3 through the shot noise. */
#define PSPEC_YLM_RTABLE_AUTO_MAX ((int64_t)96 << 30)

typedef struct {
  const void* pos;         /* device, count x 3 row-major, dtype per pos_dtype */
  int32_t pos_dtype;       /* PSPEC_POS_F64 or PSPEC_POS_F32 */
  const double* weight;    /* device, completeness weight w_c per particle, or NULL (= 1) */
  const double* nbar;      /* device, n̄ per particle, or NULL (= params.nbar) */
  int64_t count;           /* number of particles, >= 0 (randoms need > 0) */
} pspec_catalog;

typedef struct {
  double alpha, I, S;      /* as defined above */
  double W_d, W_r;         /* sums of completeness weights */
  int64_t n_nonfinite;     /* particles with a non-finite weight or nbar, or a position non-finite or
                              more than 2^40 cells from the corner (an error) */
  int64_t n_wrapped;       /* particles outside [corner, corner + L)^3, painted periodically */
} pspec_stats;

/* Device bytes a context with these parameters needs for a multipole call with up to
 * `max_kbins` bins. Returns PSPEC_EINVAL / PSPEC_EUNSUPPORTED for bad parameters. */
pspec_status pspec_workspace_size(const pspec_params* p, int32_t max_kbins, int64_t* bytes);

/* Create a context on CUDA device `device`, enqueuing on `stream` (a cudaStream_t, or NULL
 * for the legacy default stream). `workspace` is a device buffer of at least
 * pspec_workspace_size() bytes, 256-byte aligned, owned by the caller. */
pspec_status pspec_create(const pspec_params* p, int32_t device, void* stream, void* workspace,
                          int64_t workspace_bytes, int32_t max_kbins, void** ctx);
pspec_status pspec_destroy(void* ctx);

/* Step a1 + a2: FP64 catalog sums (alpha, I, S) and painting of data (+v) and randoms
 * (-alpha v) onto the mesh(es). Positions, weights and nbar are read on the device.
 * `stats` (host, nullable) is filled after a stream synchronisation, and an invalid
 * particle (see n_nonfinite) then gives PSPEC_EINVAL. With stats == NULL the call does not
 * synchronise and invalid particles are left out of the sums and the meshes. */
pspec_status pspec_paint(void* ctx, const pspec_catalog* data, const pspec_catalog* randoms,
                         pspec_stats* stats);

/* Steps a3-a6 on the painted meshes: P[i*n_kbins + b] for l = ells[i], k_mean[b] and
 * n_modes[b], all host arrays. `ells` (host) are <= the context's ell_max, any order, no
 * repeats. `k_edges` (host) has n_kbins + 1 strictly increasing, finite, >= 0 values.
 * Empty bins give NaN in P and k_mean and 0 in n_modes. Modes at or beyond the last edge are
 * never binned, and the harmonics' transforms skip x columns made only of such modes, so the
 * cost falls when the edges stop below the largest |k| of the mesh.
 * Odd l: the shell average of eq. Pell-yama (Sec. 2.1) is purely imaginary for odd l with
 * the end-point line of sight; P holds its imaginary part,
 *   4 pi/(I N_b) sum_b mult sum_m Y_lm(khat) Im[G_lm conj(F0)],
 * with Y_lm(khat) evaluated in the binning kernel (the Y table holds even l only). */
pspec_status pspec_multipoles(void* ctx, const int32_t* ells, int32_t n_ells,
                              const double* k_edges, int32_t n_kbins,
                              double* P, double* k_mean, double* n_modes);

/* As pspec_multipoles, but P, k_mean and n_modes are device buffers and the call does not
 * synchronise (capturable in a CUDA graph once the same ells/k_edges were seen before). */
pspec_status pspec_multipoles_device(void* ctx, const int32_t* ells, int32_t n_ells,
                                     const double* k_edges, int32_t n_kbins,
                                     double* P_dev, double* k_mean_dev, double* n_modes_dev);

/* Step a7: out[w*n_kbins + b] = sum_i P[i*n_kbins + b] * Lbar_{ells[i]}(mu_w, mu_{w+1}).
 * P and out are DEVICE arrays; ells and mu_edges are host arrays; the mean Legendre
 * table is built in FP64 on the host. mu_edges: n_mu + 1 increasing values in [0, 1].
 * ells must be even (an odd l gives PSPEC_EUNSUPPORTED).
 * Enqueued on `stream` without synchronising. */
pspec_status pspec_wedges(const double* P, const int32_t* ells, int32_t n_ells, int32_t n_kbins,
                          const double* mu_edges, int32_t n_mu, double* out, void* stream);

/* Splitting one catalog's multipoles across GPUs (the 2l+1 transforms of a multipole are
 * independent, Sec. 2.1). The harmonics of the requested multipoles l >= 2, listed l by l
 * (order of `ells`) and within l as m = 0, +1, -1, +2, -2, ..., form one list of
 * sum(2l+1) items. pspec_multipoles_range computes, on the painted meshes, the raw FP64 bin
 * sums of items [q0, q1) into the DEVICE array bins (1 + n_ells) x n_kbins: slot 0 holds
 * sum mult |F0|^2 when include_p0 (else zeros), slot 1 + i the sum for ells[i] (zeros for
 * l = 0 and for multipoles outside the range). Adding up the arrays of calls that cover the
 * list once (say one per GPU, then an all-reduce) and passing the sum to pspec_finalize_bins
 * (same context state, same ells and k_edges) gives what pspec_multipoles_device gives.
 * Both enqueue on the context's stream without synchronising. */
pspec_status pspec_multipoles_range(void* ctx, const int32_t* ells, int32_t n_ells, const double* k_edges,
                                    int32_t n_kbins, int32_t q0, int32_t q1, int32_t include_p0, double* bins);
pspec_status pspec_finalize_bins(void* ctx, const double* bins, const int32_t* ells, int32_t n_ells,
                                 const double* k_edges, int32_t n_kbins, double* P_dev, double* k_mean_dev,
                                 double* n_modes_dev);

/* The same multipoles (l in {0, 2, 4}) through the Cartesian decomposition that the paper
 * compares the spherical-harmonic route against (Sec. 2.1: (khat . rhat)^n expanded into the
 * monomials khat_i ... rhat_i ...; 1 + 6 + 15 = 22 transforms for l <= 4 against 1 + 5 + 9 = 15).
 * Transforms of f times each monomial rhat^q of degree 2 and 4 are binned against F0 with the
 * factors mult_q khat^q; P_2 = 5/2 (3 A_2 - B_0)/(I N_b), P_4 = 9/8 (35 A_4 - 30 A_2 + 3 B_0)/(I N_b),
 * with B_0 the l = 0 sum before the shot-noise subtraction. Equal to pspec_multipoles in
 * exact arithmetic. Needs an FP32 context created with cartesian = 1 (else PSPEC_EUNSUPPORTED);
 * outputs and synchronisation as pspec_multipoles. */
pspec_status pspec_multipoles_cartesian(void* ctx, const int32_t* ells, int32_t n_ells, const double* k_edges,
                                        int32_t n_kbins, double* P, double* k_mean, double* n_modes);

/* Transverse (mu = 0) systematics, Sec. 3.1 (host functions, FP64, no context needed).
 * pspec_transverse_response: R(mu) of eq. response, the leakage into P(k, mu) of a spike
 * P_c(k) delta(mu) reconstructed from the even multipoles up to ell_max:
 *   R(mu) = -(ell_max+1)/(2 mu) L_ell_max(0) L_{ell_max+1}(mu)  (its limit at mu = 0).
 * pspec_mu_edges_nonuniform: the ell_max/2 + 2 wedge edges 0 = mu_0 < mu_1 < ... < 1 of eq.
 * nonuniform-bins, for which the integral of L_{ell_max+1}(mu)/mu over every wedge but the
 * first vanishes, so that such a spike only enters the first wedge. mu_edges holds
 * ell_max/2 + 2 doubles (host). ell_max even, 2..16; else PSPEC_EINVAL. */
pspec_status pspec_transverse_response(int32_t ell_max, const double* mu, int32_t n, double* R);
pspec_status pspec_mu_edges_nonuniform(int32_t ell_max, double* mu_edges);

/* Wedge statistics, Sec. 4.1 (host functions, FP64).
 * pspec_wedge_lbar: the n_mu x n_ells matrix (row-major, host) of mean Legendre polynomials
 * over each wedge (eq. Lbar), the map from multipoles to wedges used by pspec_wedges.
 * pspec_wedge_gamma_kaiser: gamma_mn of eq. gamma, the angular part of the Gaussian covariance
 * of wedges built from the even multipoles 0..ell_max under the linear Kaiser model
 * (1 + beta mu^2)^2: sum_{l,l'} (2l+1)(2l'+1) Lbar_l(mu_m) Lbar_l'(mu_n) int dmu/2 L_l L_l'
 * (1 + beta mu^2)^4, into the host n_mu x n_mu array gamma (row-major). The scale factor
 * 2 P^2 / N_k of eq. trunc-Cmn is left out. Bad sizes or edges give PSPEC_EINVAL. */
pspec_status pspec_wedge_lbar(const int32_t* ells, int32_t n_ells, const double* mu_edges, int32_t n_mu,
                              double* out);
pspec_status pspec_wedge_gamma_kaiser(int32_t ell_max, const double* mu_edges, int32_t n_mu, double beta,
                                      double* gamma);

/* Batched mocks sharing one randoms catalog (the batching pattern of the mock campaigns
 * that motivate the method, Sec. 1 and Sec. 5). Needs a context created with cache_randoms = 1.
 * pspec_set_randoms paints the randoms once (unscaled) into cached meshes and keeps their
 * sums (W_r, S_r, I_r). pspec_run_batch then computes, for each of the n_mocks data catalogs
 * (host array of descriptors; device pointers inside; n_mocks <= PSPEC_MAX_BATCH), exactly
 * what pspec_paint + pspec_multipoles would give with those randoms: the data are painted,
 * mesh = data - alpha * randoms is formed on the device, and the multipoles are computed.
 * Outputs (device): P_all[mock][i][b] (n_mocks x n_ells x n_kbins), sums_all[mock] =
 * {alpha, I, S, W_d} (nullable), k_mean and n_modes (n_kbins each; the same for every mock).
 * With use_graph = 1 one mock's launch sequence is captured once as a CUDA graph (reused
 * while ells, k_edges and the paint path stay the same) and replayed per mock; the kernels
 * read the current mock from a device table and advance a device counter, so the host only
 * launches the graph. Enqueued on the context's stream; returns without synchronising. */
#define PSPEC_MAX_BATCH 4096
pspec_status pspec_set_randoms(void* ctx, const pspec_catalog* randoms);
pspec_status pspec_run_batch(void* ctx, const pspec_catalog* mocks, int32_t n_mocks, const int32_t* ells,
                             int32_t n_ells, const double* k_edges, int32_t n_kbins, double* P_all,
                             double* sums_all, double* k_mean, double* n_modes, int32_t use_graph);

/* Catalog sums without any device allocation. The paper has no counterpart: this exists
 * for callers that cannot call cudaMalloc (code that runs while a CUDA graph is being
 * captured, runtimes without a device allocator, or frameworks whose memory pool owns every
 * byte of the device). It computes what pspec_paint computes for alpha, I and S, into the
 * caller's DEVICE buffer `out` of 10 doubles: [0] W_d, [1] W_r, [2] alpha, [3] I, [4] S,
 * [5] 0, [6] 0, [7] sum_data v^2, [8] sum_randoms v^2, [9] sum_randoms nbar w_c w_fkp^2,
 * for the box, n̄ and P0 of `p` (the rest of `p` is not used). Invalid particles are left out.
 * Scratch: a fixed 64 KiB device array inside the library, held by every GPU that loads it
 * until the process exits; `nblocks` partial sums per catalog (0 = twice the SM count, at
 * most PSPEC_NOALLOC_MAX_BLOCKS; a larger value gives PSPEC_EINVAL). The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture. The address is kept for the
 * life of the process, so a device that cudaDeviceReset has reset must not be used with this
 * call again. Every call on a device shares the array, so calls that overlap on the GPU
 * (different streams, no ordering) race. The call is enqueued on `stream` and does not
 * synchronise. A CUDA error already pending on the calling thread gives PSPEC_ECUDA before
 * anything is launched (the error is left pending for its owner). */
#define PSPEC_NOALLOC_MAX_BLOCKS 1024
pspec_status pspec_catalog_sums_noalloc(const pspec_params* p, const pspec_catalog* data,
                                        const pspec_catalog* randoms, int32_t nblocks, double* out,
                                        void* stream);

/* Runtime knobs of a context and the autotuner that picks them (batching pattern: the
 * transform tiles and the paint strategy are chosen by measurement).
 *   paint_binned       1: tile-binned paint when the catalogs fit max_particles; 0: direct atomics
 *   ylm_harmonics      harmonics per block of the Y_lm-weighted z pass (>= 1)
 *   bin_blocks_per_sm  persistent blocks per SM of the combine/binning passes (0: occupancy limit)
 *   tile_y             0: the compiled y-pass tile; 1: half as many columns per block
 * pspec_autotune paints the given catalogs and times pspec_multipoles_device for candidate
 * settings (reps timed runs each, CUDA events on the context's stream), keeps the fastest
 * and returns it in *best. It synchronises the stream. */
typedef struct {
  int32_t paint_binned;
  int32_t ylm_harmonics;
  int32_t bin_blocks_per_sm;
  int32_t tile_y;
} pspec_tuning;
pspec_status pspec_get_tuning(void* ctx, pspec_tuning* t);
pspec_status pspec_set_tuning(void* ctx, const pspec_tuning* t);
pspec_status pspec_autotune(void* ctx, const pspec_catalog* data, const pspec_catalog* randoms,
                            const int32_t* ells, int32_t n_ells, const double* k_edges, int32_t n_kbins,
                            int32_t reps, pspec_tuning* best);

/* Plan facts for tests and reports. */
typedef struct {
  int32_t nmesh, precision, ell_max;
  int32_t tile_y, tile_x, tile_bin, rows_z;   /* FFT tile shapes chosen */
  int32_t group_max;                          /* spectra buffered per group launch */
  int32_t bin_ctas;                           /* persistent CTAs of the binning passes */
  int64_t sh_transforms;                      /* sum over requested l of 2l+1 (paper's count) */
  int64_t transforms_executed;                /* 3-D transforms of the last multipoles call */
  int64_t kernel_launches;                    /* cumulative kernels launched by this context */
  double model_bytes_last;                    /* algorithmic HBM bytes of the last paint+multipoles */
  int64_t ylm_table_bytes;                    /* Y_lm(khat) table held (0: evaluated per mode) */
  int64_t cartesian_table_bytes;              /* Cartesian k-space factors held (0: none) */
  int64_t ylm_rtable_bytes;                   /* Y_lm(rhat) table held (0: evaluated per node) */
} pspec_plan_info;
pspec_status pspec_get_plan_info(void* ctx, pspec_plan_info* info);

/* Per-kernel-class timing with CUDA events on the context's stream, for the benchmark.
 * While enabled, each launch is bracketed by events; pspec_kernel_times returns, per
 * class, the number of launches, the summed milliseconds and the algorithmic bytes. */
enum { PSPEC_K_SUMS = 0, PSPEC_K_PAINT, PSPEC_K_FFT_Z, PSPEC_K_FFT_Y, PSPEC_K_FFT_X,
       PSPEC_K_COMBINE, PSPEC_K_YLM_Z, PSPEC_K_BIN_X, PSPEC_K_C2R_Z, PSPEC_K_FINAL,
       PSPEC_K_OTHER, PSPEC_K_COUNT };
pspec_status pspec_set_profiling(void* ctx, int32_t enable);
pspec_status pspec_kernel_times(void* ctx, int64_t* launches, double* ms, double* bytes);
const char* pspec_kernel_name(int32_t k);

const char* pspec_strerror(pspec_status s);
const char* pspec_last_error(void* ctx);
/* Library version string and the compiled-in architecture. */
const char* pspec_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PSPEC_H */

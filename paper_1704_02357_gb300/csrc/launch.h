// Host-side launchers of the libpspec kernels (internal; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"
#include "pspec.h"

namespace pspec {

// Layout facts every pass needs.
struct Geo {
  int N;   // mesh side
  int NH;  // stored kz per row (N/2; the kz = N/2 plane is never stored)
};

// Slots of the FP64 bin sums: [slot][kbin].
enum { SLOT_P0 = 0, SLOT_ELL0 = 1 };
// Layout of the derived catalog quantities (device doubles).
enum { D_WD = 0, D_WR, D_ALPHA, D_I, D_S, D_NONFINITE, D_WRAPPED, D_SD, D_SR, D_IR, D_COUNT = 16 };
constexpr int kSumVals = 4;  // per-block partial: w_c, v^2, nbar w_c w_fkp^2, spare

struct PaintArgs {
  const void* pos;
  int pos_f32;
  const double* weight;
  const double* nbar;
  int64_t count;
  double corner[3];
  double inv_cell;      // N / L
  double P0;
  double nbar_default;
  double wf_default;    // FKP weight for nbar_default
};

struct BinArgs {
  const int32_t* bin_of_n2;  // bin index of |n|^2, or -1
  int nk;
  double* bins;              // [slots][nk] FP64 sums, added to with atomics
};

// a1: per-block partial sums of one weighted catalog; final combine into `derived`.
// When neither catalog carries weight or nbar arrays the closed forms are used instead.
void launch_catalog_partials(const PaintArgs& a, double* partials, int nblocks, cudaStream_t s);
void launch_catalog_final(const double* part_d, int nb_d, const double* part_r, int nb_r, double* derived,
                          cudaStream_t s);
void launch_derive_uniform(int64_t n_d, int64_t n_r, double wf, double nbar, double* derived, cudaStream_t s);

// a2: scatter-add painting; counts invalid and out-of-box particles into derived.
template <typename T>
void launch_paint(const PaintArgs& a, int window, int interlaced, int is_randoms, double* derived, T* mesh1,
                  T* mesh2, int N, int nblocks, cudaStream_t s);

// Transform passes (E = register elements per thread: 8, or 24 for N = 3*2^a).
// Tables: tw_half (L = N/2), tw_full (L = N), twr (exp(-2 pi i k/N), k < N/2).
template <typename T>
void launch_r2c_z(const T* in, cx<T>* out, const Geo& g, const FftPlan& pz, int E, const cx<T>* tw_half,
                  const cx<T>* twr, int rows, cudaStream_t s);
template <typename T>
void launch_c2r_z(const cx<T>* in, T* out, const Geo& g, const FftPlan& pz, int E, const cx<T>* tw_half,
                  const cx<T>* twr, int rows, T scale, cudaStream_t s);
template <typename T>
void launch_ylm_r2c_z(const T* f, cx<T>* out, int64_t spec_stride, int ell, int h0, int M, const Geo& g,
                      const FftPlan& pz, int E, const cx<T>* tw_half, const cx<T>* twr, const T* axis_pos, int rows,
                      int threads, cudaStream_t s);
template <typename T>
void launch_fft_y(cx<T>* data, int64_t spec_stride, int nspec, const Geo& g, const FftPlan& pf, int E,
                  const cx<T>* tw_full, int tw, int dir, cudaStream_t s);
template <typename T>
void launch_fft_x(const cx<T>* in, cx<T>* out, const Geo& g, const FftPlan& pf, int E, const cx<T>* tw_full, int tw,
                  int dir, cudaStream_t s);
template <typename T>
void launch_combine_x(const cx<T>* B, cx<T>* F0, const Geo& g, const FftPlan& pf, int E, const cx<T>* tw_full, int tw,
                      int interlaced, int compensate, int roundtrip, const cx<T>* phase_axis, const T* invw_axis,
                      const BinArgs& ba, int ctas, cudaStream_t s);
template <typename T>
void launch_bin_x(const cx<T>* G, int64_t spec_stride, int ell, int h0, int M, const cx<T>* F0, const Geo& g,
                  const FftPlan& pf, int E, const cx<T>* tw_full, int tw, int slot, const BinArgs& ba, int ctas,
                  cudaStream_t s);

// Mode counts: cnt[|n|^2] over binnable modes (once per plan), then N_b and sum |k| per bin.
void launch_mode_counts(const Geo& g, unsigned int* cnt, int nsm, cudaStream_t s);
void launch_bin_counts(const unsigned int* cnt, const double* kmag, const int* lo, const int* hi, int nk,
                       double* nmodes, double* ksum, cudaStream_t s);

// a6: bin sums -> P_l, k_mean, n_modes (device doubles).
void launch_finalize(const double* bins, const double* nmodes, const double* ksum, int nk, const int32_t* ells,
                     int n_ells, const double* derived, double* P, double* k_mean, double* n_modes, cudaStream_t s);

// a7: out[w][b] = sum_i P[i][b] lbar[i][w].
constexpr int kMaxWedgeTab = 9 * 64;
struct WedgeTab {
  double lbar[kMaxWedgeTab];  // [i * n_mu + w]
};
void launch_wedges(const double* P, int n_ells, int nk, int n_mu, const WedgeTab& t, double* out, cudaStream_t s);

// Shared-memory sizes and persistent CTA counts (which: 0 combine, 1 bin).
size_t smem_rows(int L, int rows, size_t csz);
template <typename T> size_t smem_cols(const Geo& g, int tw);
template <typename T> size_t smem_ylm_z(const Geo& g, int E, int M, int rows, int threads);
template <typename T> size_t smem_combine(const Geo& g, int E, int tw, int nk);
template <typename T> size_t smem_bin_x(const Geo& g, int E, int tw, int nk);
template <typename T> int persistent_ctas(int which, const Geo& g, int E, int tw, int nk, int nsm);

// Y_lm coefficient tables (FP64-built) into constant memory of the current device.
cudaError_t upload_ylm_tables(cudaStream_t s);

}  // namespace pspec

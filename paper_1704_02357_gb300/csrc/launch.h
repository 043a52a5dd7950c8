// Host-side launchers of the libpspec kernels (internal; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"
#include "pspec.h"

namespace pspec {

// Layout facts every pass needs.
struct Geo {
  int N;       // mesh side
  int NH;      // stored kz per row (N/2; the kz = N/2 plane is never stored)
};

// Slots of the per-CTA partial bins: [cta][slot][kbin].
enum { SLOT_NMODES = 0, SLOT_KSUM = 1, SLOT_P0 = 2, SLOT_ELL0 = 3 };
// Layout of the derived catalog sums (device doubles).
enum { D_WD = 0, D_WR, D_ALPHA, D_I, D_S, D_NONFINITE, D_WRAPPED, D_SD, D_SR, D_IR, D_COUNT = 16 };
constexpr int kSumVals = 6;   // per-catalog partial: w_c, v^2, nbar w_c w_fkp^2, nonfinite, wrapped, spare

struct PaintArgs {
  const void* pos;
  int pos_f32;
  const double* weight;
  const double* nbar;
  int64_t count;
  double corner[3];
  double cell;
  double P0;
  double nbar_default;
};

// a1: per-block partial sums of one catalog; final combine into `derived`.
void launch_catalog_partials(const PaintArgs& a, int nmesh, double* partials, int nblocks, cudaStream_t s);
void launch_catalog_final(const double* part_d, int nb_d, const double* part_r, int nb_r,
                          double* derived, cudaStream_t s);

// a2: scatter-add painting. sign: +1 data, -alpha (read from derived) randoms.
template <typename T>
void launch_paint(const PaintArgs& a, int window, int interlaced, int is_randoms, const double* derived,
                  T* mesh1, T* mesh2, int N, int nblocks, cudaStream_t s);

// Transform passes. Tables: tw_half (L = N/2), tw_full (L = N), twr (exp(-2 pi i k/N), k < N/2).
template <typename T>
void launch_r2c_z(const T* in, cx<T>* out, const Geo& g, const FftPlan& pz, const cx<T>* tw_half,
                  const cx<T>* twr, int rows, cudaStream_t s);
template <typename T>
void launch_ylm_r2c_z(const T* f, cx<T>* out, int64_t spec_stride, int ell, int h0, int M,
                      const Geo& g, const FftPlan& pz, const cx<T>* tw_half, const cx<T>* twr,
                      const T* axis_pos, int rows, cudaStream_t s);
template <typename T>
void launch_fft_y(cx<T>* data, int64_t spec_stride, int nspec, const Geo& g, const FftPlan& pf,
                  const cx<T>* tw_full, int tw, int dir, cudaStream_t s);
template <typename T>
void launch_fft_x(const cx<T>* in, cx<T>* out, const Geo& g, const FftPlan& pf, const cx<T>* tw_full,
                  int tw, int dir, cudaStream_t s);
struct BinTabs {
  const int32_t* bin_of_n2;  // bin index of |n|^2, or -1
  const double* kmag_of_n2;  // |k| of |n|^2
  int nk;
  int nslots;
  double* partials;          // [ctas][nslots][nk]
  int ctas;
};
template <typename T>
void launch_combine_x(const cx<T>* B, cx<T>* F0, const Geo& g, const FftPlan& pf, const cx<T>* tw_full,
                      int tw, int interlaced, int compensate, int roundtrip, const cx<T>* phase_axis,
                      const T* invw_axis, const BinTabs& bt, cudaStream_t s);
template <typename T>
void launch_bin_x(const cx<T>* G, int64_t spec_stride, int ell, int h0, int M, const cx<T>* F0,
                  const Geo& g, const FftPlan& pf, const cx<T>* tw_full, int tw, int slot,
                  const BinTabs& bt, cudaStream_t s);
template <typename T>
void launch_c2r_z(const cx<T>* in, T* out, const Geo& g, const FftPlan& pz, const cx<T>* tw_half,
                  const cx<T>* twr, int rows, T scale, cudaStream_t s);

// a6: per-CTA partials -> P_l, k_mean, n_modes (device doubles).
void launch_finalize(const double* partials, int ctas, int nslots, int nk, const int32_t* ells_slot,
                     int n_ells, const double* derived, double* P, double* k_mean, double* n_modes,
                     cudaStream_t s);

// a7: out[w][b] = sum_i P[i][b] lbar[i][w].
constexpr int kMaxWedgeTab = 9 * 64;
struct WedgeTab {
  double lbar[kMaxWedgeTab];  // [i * n_mu + w]
};
void launch_wedges(const double* P, int n_ells, int nk, int n_mu, const WedgeTab& t, double* out,
                   cudaStream_t s);

// Occupancy-derived CTA counts for the persistent binning passes.
template <typename T> int bin_x_ctas(const Geo& g, int tw, int nsm, int nk_max);
template <typename T> int combine_x_ctas(const Geo& g, int tw, int nsm, int nk_max);
template <typename T> size_t smem_combine(const Geo& g, int tw, int nk);
template <typename T> size_t smem_fft_y(const Geo& g, int tw);
template <typename T> size_t smem_bin_x(const Geo& g, int tw);
template <typename T> size_t smem_ylm_z(const Geo& g, int M, int rows);

// Y_lm coefficient tables (FP64-built) into constant memory of the current device.
cudaError_t upload_ylm_tables(cudaStream_t s);

}  // namespace pspec

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
// D_FIX: the fixed-point scale 2^S of the exact (tile-binned) paint for the catalogs painted
// together by pspec_paint (or a mock's data alone).
enum { D_WD = 0, D_WR, D_ALPHA, D_I, D_S, D_NONFINITE, D_WRAPPED, D_SD, D_SR, D_IR, D_FIX, D_COUNT = 16 };
constexpr int kSumVals = 4;  // per-block partial: w_c, v^2, nbar w_c w_fkp^2, |v|

// A catalog as a device-side descriptor (batched mocks: the kernels of one captured graph
// read the current mock's catalog from a table indexed by a device counter).
struct DevCat {
  const void* pos;
  const double* weight;
  const double* nbar;
  long long count;
  int pos_f32;
  int pad;
};

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
  const DevCat* dc;     // when set, pos/weight/nbar/count come from dc[*cur]
  const int* cur;
};

struct BinArgs {
  const int32_t* bin_of_n2;  // bin index of |n|^2, or -1
  int nk;
  double* bins;              // [slots][nk] FP64 sums, added to with atomics
  const void* permode_w;     // compensation applied per mode in the binning (cx<T> per-axis table), or nullptr
  int odd;                   // odd l: bin Y Im[G conj(F0)] instead of Y Re[G conj(F0)]
  // binning pass: the x-pass tiles (j * (N/2/TW) + kz0/TW) holding a binned mode, in order
  // (a tile whose columns all have ny^2 + kz^2 beyond the last bin is left out)
  const int32_t* xtiles;
  int n_xtiles;
};

// a1: per-block partial sums of one weighted catalog; final combine into `derived`.
// When neither catalog carries weight or nbar arrays the closed forms are used instead.
void launch_catalog_partials(const PaintArgs& a, double* partials, int nblocks, cudaStream_t s);
// `fix` (nullable): where to store the exact paint's fixed-point scale for both catalogs.
void launch_catalog_final(const double* part_d, int nb_d, const double* part_r, int nb_r, double* derived,
                          cudaStream_t s, double* fix = nullptr);
void launch_derive_uniform(int64_t n_d, int64_t n_r, double wf, double nbar, double* derived, cudaStream_t s);

// Batched mocks: randoms sums kept from pspec_set_randoms (W_r, S_r, I_r), the data sums of
// the current mock combined with them; mesh -= alpha * cached randoms mesh; counter += 1.
void launch_catalog_final_cached(const double* part_d, int nb_d, const double* rsums, double* derived,
                                 cudaStream_t s);
void launch_randoms_sums(const double* part_r, int nb_r, double* rsums, cudaStream_t s);
void launch_axpy_randoms(float* mesh, const float* rmesh, int64_t n, const double* derived, cudaStream_t s);
void launch_axpy_randoms(double* mesh, const double* rmesh, int64_t n, const double* derived, cudaStream_t s);
// Destinations of a batch's per-mock results, read by the kernel from device memory (they are
// uploaded before every batch), so that a captured graph replays into the current call's buffers.
struct BatchOut {
  double* P_all;
  double* sums_all;
};
void launch_batch_outputs(const double* P, int n_ells, int nk, const double* derived, const int* cur,
                          const BatchOut* out, cudaStream_t s);
void launch_advance(int* cur, cudaStream_t s);

// a2: scatter-add painting; counts invalid and out-of-box particles into derived.
// is_randoms: 0 data (+v), 1 randoms (-alpha v), 2 randoms unscaled (+v, cached meshes).
template <typename T>
void launch_paint(const PaintArgs& a, int window, int interlaced, int is_randoms, double* derived, T* mesh1,
                  T* mesh2, int N, int nblocks, cudaStream_t s);

// a2, tile-binned (FP32 meshes), exact: prep (records + per-tile counts, a particle counted for
// every 16^3 tile its footprint touches) per catalog, scan, scatter into tile order, then one
// block per tile sums its cells in 64-bit fixed point (scale 2^S at `fix`) and stores every
// cell of the tile once (no mesh clearing needed). Tile side kPaintTile divides N. The sorted
// copy holds up to 8 records per particle (kPaintRecordsMax).
constexpr int kPaintTile = 16;
constexpr int kPaintRecordsMax = 8;
struct TileArgs {
  unsigned* cnt;     // [ntiles] records per tile (cleared before prep)
  unsigned* off;     // [ntiles] exclusive prefix of cnt
  unsigned* cursor;  // [ntiles] scatter cursors
  uint4* rec;        // [particles] records in input order
  unsigned* tile_of; // [particles] first tile of each record (all ones: left out)
  uint4* sorted;     // [kPaintRecordsMax * particles] records in tile order
};
void launch_ptile_prep(const PaintArgs& a, int window, int interlaced, int is_randoms, double* derived,
                       const TileArgs& ta, int64_t offset, int N, int nblocks, cudaStream_t s);
void launch_ptile_scan(const TileArgs& ta, int ntiles, cudaStream_t s);
void launch_ptile_scatter(const TileArgs& ta, int64_t total, const DevCat* dc, const int* cur, int N, int nblocks,
                          cudaStream_t s);
void launch_ptile_paint(const TileArgs& ta, int window, int interlaced, float* m1, float* m2, int N,
                        const double* fix, cudaStream_t s);

// Transform passes, one table of launchers per supported mesh side N (pass_*.cu).
// Tables: tw_half (L = N/2), tw_full (L = N), twr (exp(-2 pi i k/N), k < N/2).
// Shapes fixed per N at compile time:
//   col_tile(N): kz columns per y/x tile, a power of two dividing N/2 with at most 512
//                threads (N/E per column) and at most 16 columns;
//   z_rows(N):   rows per block of the plain z passes, a power of two dividing N^2 with at
//                most 512 threads (N/(2E) per row).
constexpr int elems_per_thread(int N) { return N % 3 == 0 ? 24 : 8; }
constexpr int col_tile(int N) {
  const int tc = N / elems_per_thread(N);
  int cap = 512 / tc < 16 ? 512 / tc : 16, tw = 1;
  // N * TW <= 4096 keeps two FP64 tiles (binning pass) plus the bins within shared memory
  while (tw * 2 <= cap && (N / 2) % (tw * 2) == 0 && N * tw * 2 <= 4096) tw *= 2;
  return tw;
}
// Elements per thread in the z passes (rows of N/2 complex points): 16 where a row splits into
// radix-16 stages (one exchange fewer than radix 8 for 256 points), else as elsewhere.
constexpr int z_elems(int N) { return N % 3 == 0 ? 24 : (N / 2 >= 128 ? 16 : 8); }
constexpr int z_rows(int N) {
  const int tz = (N / 2) / z_elems(N);
  int cap = 512 / tz, r = 1;
  while (r * 2 <= cap && ((long long)N * N) % (r * 2) == 0) r *= 2;
  return r;
}

// Threads of one block of the Y_lm-weighted z pass (harmonics x rows x threads per row) and
// the resident blocks per SM its register allocation must allow (0: no requirement). The
// unrolled l = 4 kernel launches at most 288 threads (9 x 16 x 2 at N = 512) and l = 2 at most
// 160 (5 x 16 x 2); capping them there keeps them within 56 registers, so that 4 and 7 blocks
// share an SM instead of 3 and 6.
__host__ __device__ constexpr int ylm_thread_cap(int lt) { return lt == 4 ? 288 : (lt == 2 ? 160 : 512); }
__host__ __device__ constexpr int ylm_min_blocks(int lt, bool xp = false) {
  return xp ? (lt == 4 ? 2 : (lt == 2 ? 4 : 0)) : (lt == 4 ? 4 : (lt == 2 ? 7 : 0));
}

// Twiddle and phase tables hold ux<T> entries (FP32: {cos, sin, 1/|w| - 1, 0}); the
// compensation table holds cx<T> {1/W_d rounded, its relative rounding error}.
// Y_lm(khat) table of the FP32 binning pass: harmonic slots of l = 2, 4, ..., l_max in order,
// 2l+1 each (h order of the harmonics), every slot one value per stored mode, one contiguous
// block of N x tw values per x tile (j, kz tile) of the binning pass, rows i.
__host__ __device__ constexpr int ytab_base(int ell) {
  int b = 0;
  for (int l = 2; l < ell; l += 2) b += 2 * l + 1;
  return b;
}
void launch_ytab_build(float* ytab, int N, int tw, int ell_max, int nsm, cudaStream_t s);
// Y_lm(rhat) of every mesh node for the Y-weighted z pass (FP32 contexts): the same harmonic
// slots as the Y_lm(khat) table, every slot one value per node [i][j][k], built in FP64 and
// rounded once. Evaluated in FP32 per node instead, the weights carry errors that are coherent
// over the sphere (position rounding, the recurrence and the complex power); through them the
// shot noise leaks into P_l, ~1e-4 of P_14 and ~2e-5 of a small P_4 at 512^3.
struct RGeo {
  double corner[3], H, observer[3];
};
void launch_rtab_build(float* rtab, int N, int ell_max, const RGeo& g, int nsm, cudaStream_t s);
// Cartesian k-space factors mult_q khat^q of every stored mode, q = 0..20 (kCartItems slots).
void launch_ctab_build(float* ctab, int N, int tw, int nsm, cudaStream_t s);

// Launchers with an `xp` argument run the exact-add FP32 variant of their kernel (xp_engine.cuh)
// when it is nonzero and T is float; FP64 ignores it.
template <typename T> struct PassTable {
  int N, E, tw, rows_z, tz;
  int tz_xp;  // threads per row of the exact-add z passes
  void (*r2c_z)(const T*, cx<T>*, const ux<T>*, const ux<T>*, cudaStream_t);
  void (*c2r_z)(const cx<T>*, T*, const ux<T>*, const ux<T>*, T, int, cudaStream_t);
  // ..., rows, Y_lm(rhat) table slot of the group's first harmonic (FP32) or nullptr, xp
  void (*ylm_z)(const T*, cx<T>*, int64_t, int, int, int, const ux<T>*, const ux<T>*, const T*, int, const float*,
                int, cudaStream_t);
  size_t (*smem_ylm)(int, int);
  // ..., dir, tile variant, n2_cut (outputs with ny^2 + kz^2 >= n2_cut are not stored), xp
  void (*fft_y)(cx<T>*, int64_t, int, const ux<T>*, int, int, int, int, cudaStream_t);
  void (*fft_x)(const cx<T>*, cx<T>*, const ux<T>*, int, int, cudaStream_t);
  void (*combine_x)(const cx<T>*, cx<T>*, const ux<T>*, int, int, int, const ux<T>*, const cx<T>*, const BinArgs&,
                    int, cudaStream_t);
  void (*bin_x)(const cx<T>*, int64_t, int, int, int, const cx<T>*, const ux<T>*, int, const BinArgs&, int,
                const float*, int, cudaStream_t);  // ..., table slot of the group's first harmonic or nullptr, xp
  int (*ctas)(int, int, int, int);  // (which: 0 combine, 1 bin, 2 pipelined FP32 bin; nk; SMs; xp) -> persistent blocks
  size_t (*smem_combine)(int);
  size_t (*smem_bin)(int);
  size_t (*smem_bin_pipe)(int);
};
template <typename T, int N> const PassTable<T>* pass_table_n();
// nullptr when N is not a supported mesh side.
template <typename T> const PassTable<T>* pass_table(int N);
// Y_lm recurrence coefficients (built in FP64 on the host), passed to kernels by value.
template <typename T> const YTab<T>& host_ytab();

// Mode counts: cnt[|n|^2] over binnable modes (once per plan), then N_b and sum |k| per bin.
void launch_mode_counts(const Geo& g, unsigned int* cnt, int nsm, cudaStream_t s);
void launch_bin_counts(const unsigned int* cnt, const double* kmag, const int* lo, const int* hi, int nk,
                       double* nmodes, double* ksum, cudaStream_t s);

// a6: bin sums -> P_l, k_mean, n_modes (device doubles).
void launch_finalize(const double* bins, const double* nmodes, const double* ksum, int nk, const int32_t* ells,
                     int n_ells, const double* derived, double* P, double* k_mean, double* n_modes, cudaStream_t s,
                     int cartesian = 0);

// a7: out[w][b] = sum_i P[i][b] lbar[i][w].
constexpr int kMaxWedgeTab = 9 * 64;
struct WedgeTab {
  double lbar[kMaxWedgeTab];  // [i * n_mu + w]
};
void launch_wedges(const double* P, int n_ells, int nk, int n_mu, const WedgeTab& t, double* out, cudaStream_t s);

}  // namespace pspec

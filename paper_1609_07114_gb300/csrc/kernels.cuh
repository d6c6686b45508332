// Device kernels of the time-marching hot path (sm_103a).
//
// One time step n -> n+1 (Sec. IV-C) is two launches:
//   yee_step   : coarse Hz^{n+1/2} (Eq. (5)) and coarse E^{n+1} (Eq. (3))
//                fused per tile, plus the source current on its edges;
//   rom_post   : every embedded model's run-time map (Eq. (23)),
//                [y; x~]^{n+1} = P [y; x~]^n + Q h^{n+1/2}, and the probes.
// Fields are ping-ponged between two buffers (read p, write 1-p), so tiles
// can recompute their one-cell H halo without racing their neighbours.
//
// Memory layout per simulation: Ex, Ey, Hz each (ny+1) rows x pitch floats,
// row-major, pitch a multiple of 128 floats (512 B) and > nx; cell materials
// as float2 {eps0 eps_r / dt + sigma / 2, sigma}, the first component set to
// -1 for cells covered by a reduced model.  An E edge is updated only if both its
// cells are coarse cells and it is not on the PEC wall.
//
// Sparse materials: a simulation's most frequent cell material is its
// background mbg.  One bit per (row, 128-column strip) says whether any cell
// of the strip, or the cell just left of it, differs from mbg; the stencil
// reads the materials of flagged strip rows only (a vacuum grid with sparse
// scatterers moves 24 B per cell-step instead of 32).
#pragma once

#include <cstdint>

namespace fdtdrom {

// A stencil CTA covers kCtaCols columns x (per-simulation) tile rows.  Lanes
// own V = 2 or 4 consecutive columns, so a warp strip is 32 V columns and a
// CTA has kCtaCols / (32 V) warps.
constexpr int kCtaCols = 512;

struct SimDev {
  float* ex[2];
  float* ey[2];
  float* hz[2];
  const float2* mat;
  const uint32_t* mbits;  // [(ny + 31) / 32][nstrip]: bit (j & 31) of word (j / 32, strip)
  float2 mbg;             // background material
  int nx, ny, pitch, nstrip;
  float chx;   // dt / (mu0 dy):  Hz += chx (Ex_{j+1} - Ex_j)
  float chy;   // dt / (mu0 dx):  Hz -= chy (Ey_{i+1} - Ey_i)
  float rdy;   // 1/dy: Ex += cb (Hz_j - Hz_{j-1}) / dy
  float rdx;   // 1/dx: Ey -= cb (Hz_i - Hz_{i-1}) / dx
  float rdy2;  // 2/dy, 2/dx: the same products from r = cb / 2
  float rdx2;
  float* exm;  // two-step launches that keep every step's E (the gradient's
  float* eym;  // recomputation): E^{n+1} between the sub-steps; else null
};

struct TileWork {   // one CTA of yee_step: columns [x0, x0 + kCtaCols), rows [y0, y1)
  int sim, x0, y0, y1;
};

struct SrcEdge {    // one driven edge
  int sim, comp, i, j;
  int src;          // index of the waveform
  int pad[3];
};

struct RomInstDev {
  const float* M;     // n x ld row-major: [P | Q | 0], ld = roundup(n + ny, 4)
  float* state[2];    // [y; x~] (ld floats: [y; x~; h; 0]), ping-ponged with the fields
  float* state_mid;   // two-step path, maps outside the tile: [y; x~; h]^{n+1} between the sub-steps
  const int* y_edge;  // ny: (comp << 30) | (j * pitch + i)
  const int* h_cell;  // ny: j * pitch + i
  int n, ny, ld, sim;
};

constexpr int kRomRowsPerCta = 8;   // one row per warp

// Simulations that share one coupled map step it as one GEMM:
// [S'] = [P | Q] [S; H] with one column per simulation (CTA: 8 rpw rows x
// 32 columns).
struct GemmGroupDev {
  const float* M;       // [P | Q | 0], n x ld
  int n, ny, ld, B;     // B instances, listed at ginst[inst_off ...]
  int inst_off, rpw;    // rpw: rows per warp of the CTA tiles (1 or 2)
  int pad1, pad2;
};

struct GemmWork {
  int group, r0, c0, pad;
};

struct RomWork {    // one CTA of rom_post: rows [row0, row1) of one instance
  int inst, row0, row1, pad;
};

// Convolutional PML of one simulation: per coordinate the coefficients
// {b, a, 1/kappa} of the stretched differences ([3][len] arrays, at the
// positions where each difference is taken: x-arrays of Hz/Ex over nx
// columns, of Ey over nx + 1; y-arrays of Hz/Ey over ny rows, of Ex over
// ny + 1).
struct PmlSimDev {
  const float* xh;
  const float* yh;
  const float* xe;
  const float* ye;
  int nxh, nyh, nxe, nye;   // array lengths
  float dtmu;               // dt / mu0
  int pad;
};

struct EnergyInstDev {  // storage-function data of one embedded model
  const double* R;      // q x q: R~ of Eq. (12) at the run dt
  const double* c1;     // ny: 1/2 Dl Dl' eps_b  (interface half cells)
  const double* c2;     // ny: dt/2 * (Dl G^T)_k
  int q, sim, pad0, pad1;
};

struct RunDev {
  long long base;            // step index, relative to the run start, of chunk step 0
  long long nsteps;
  const float* const* waves; // per source: device samples J(t^{n+1/2})
  const int2* src_range;     // per yee_step CTA: [begin, end) into src_edges
  const SrcEdge* src_edges;
  float* probe_out;          // [nsteps][nprobe]
  const int* probe_sim;
  const int* probe_cell;     // j * pitch + i
  int nprobe;
  int ndft;                  // DFT monitors x frequencies (0: none)
  // Running DFT of Hz at monitor cells (frequency responses): the step
  // index of the context at the run start, per frequency f dt (cycles per
  // step), per monitor its simulation and cell, and FP64 accumulators
  // sum_n Hz^{n+1/2} exp(-i 2 pi f (n + 1/2) dt), [monitor][frequency].
  long long step0;
  const double* dft_fdt;
  const int* dft_sim;
  const int* dft_cell;
  double2* dft_acc;
  int nfreq;
  int pf1;                   // one-step stencil: rows prefetched into L1 ahead of its loads (0: none)
  unsigned* status;          // device word: bit 0 = a bounded wait in a kernel gave up
};

}  // namespace fdtdrom

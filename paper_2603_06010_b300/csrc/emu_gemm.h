// FP64-accurate split products on the tensor cores (emu_gemm.cu) and the
// tensor-core factor built on them (factor_tc.cu).
#pragma once
#include "td_internal.h"

namespace td {

constexpr int EK = 128;   // contraction length of one split product (and the factor's block size)

struct EmuProb {         // D = alpha A B^T + beta D over K = EK
  CUtensorMap mapA;      // A slices [ns][rows][EK] bf16, box {32, 128, ns}
  CUtensorMap mapB;      // B slices [ns][rows][EK] bf16, box {32, 64, ns}
  const int* ea;         // per A row: the power of two of its slices
  const int* eb;         // per B row
  double* C;             // D(i, j) at C[i + j ldc]
  int64_t ldc;
  double alpha, beta;    // beta == 0: D is written without being read
  int a_row0, b_row0;    // first A / B operand row of the problem
  int m_tiles, n_tiles;  // 128-row and 64-column output tiles
  int lower;             // 1: square output, only the tiles that meet the lower triangle
  int tile_begin;        // first tile of this problem in the launch's tile list
};

struct EmuParams {
  EmuProb p[2];
  int nprob;
  int total_tiles;
};

struct EmuSplitJob {     // operand rows -> slices [ns][rows_alloc][EK] and exponents
  const double* src;     // value k of row r at src[r rs + k ks]
  int64_t rs, ks;
  int rows;              // rows to split
  int rows_alloc;        // row extent of dst (slice stride)
  __nv_bfloat16* dst;
  int* e;                // [rows]: value = 2^e sum_s slice_s
  int ns;
  int block0;            // first CTA of this job
};

struct EmuSplitParams {
  EmuSplitJob job[3];
  int njobs;
  int total_blocks;
};

inline int emu_tiles(const EmuProb& q) { return q.lower ? q.m_tiles * (q.m_tiles + 1) : q.m_tiles * q.n_tiles; }

cudaError_t launch_emu_split(const EmuSplitParams& P, cudaStream_t st);
// max_ctas > 0 caps the persistent grid (to leave SMs to a kernel on another stream)
cudaError_t launch_emu_gemm(const EmuParams& P, int ns, DevStatus* status, int64_t limit_ns, cudaStream_t st,
                            int max_ctas = 0);

}  // namespace td

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
  const void* src;       // value k of row r at src[r rs + k ks]: double, or float with src_f32
  int64_t rs, ks;
  int rows;              // rows to split
  int rows_alloc;        // row extent of dst (slice stride)
  __nv_bfloat16* dst;
  int* e;                // [rows]: value = 2^e sum_s slice_s
  int ns;
  int block0;            // first CTA of this job
  int src_f32;           // 1: the source holds FP32 values
  int rows_valid;        // rows at or beyond this one split as zero (not read)
  int lower;             // 1: value k of row r < EK is zero for k > r (a diagonal block's upper part)
  int k_valid;           // values k >= k_valid are zero (not read)
};

struct EmuSplitParams {
  EmuSplitJob job[3];
  int njobs;
  int total_blocks;
};

inline int emu_tiles(const EmuProb& q) { return q.lower ? q.m_tiles * (q.m_tiles + 1) : q.m_tiles * q.n_tiles; }

struct SliceBuf {          // operand slices [ns][rows][EK] and exponents [rows]
  __nv_bfloat16* v = nullptr;
  int* e = nullptr;
  int rows = 0;
  CUtensorMap boxA, boxB;  // 128-row (A operand) and 64-row (B operand) boxes
};
td_status slice_buf(SliceBuf& b, int rows, int ns);
void free_slice_buf(SliceBuf& b);
// one split job (rows of src, value k of row r at src[r rs + k ks]); src_f32:
// FP32 source; rows_valid: rows from it on split as zero; lower: zero above
// the diagonal of the first EK rows
void add_split_job(EmuSplitParams& P, const void* src, int64_t rs, int64_t ks, int rows, SliceBuf& dst, int ns,
                   bool src_f32 = false, int rows_valid = -1, bool lower = false, int k_valid = EK);
// one product D = alpha A B^T + beta D over 128-row x 64-column tiles
void add_product(EmuParams& P, const SliceBuf& A, const SliceBuf& B, double* C, int64_t ldc, double alpha,
                 double beta, int m_tiles, int n_tiles, bool lower, int a_row0 = 0, int b_row0 = 0);

cudaError_t launch_emu_split(const EmuSplitParams& P, cudaStream_t st);
// max_ctas > 0 caps the persistent grid (to leave SMs to a kernel on another stream)
cudaError_t launch_emu_gemm(const EmuParams& P, int ns, DevStatus* status, int64_t limit_ns, cudaStream_t st,
                            int max_ctas = 0);

}  // namespace td

// Host-side construction of the H-matrix approximation of the L1 time matrix R.
//
// Section 2 defines R (Eq. elements_matrix_R) on the graded mesh t_m = T (m/M)^gamma;
// Section 3 builds its H-matrix form: index bisection of {1..M}, the admissibility condition
// of Definition 3.1, Taylor degenerate-kernel factors (Eqs. A_elements, B_elements).  On top
// of the paper's construction this builder recompresses each Taylor block (Householder QR of
// both factors + SVD of the small core) to a block-relative tolerance, and flattens the
// block tree into per-leaf-row panels that the CUDA kernels walk in time order.
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector>

namespace fhmg {

struct RkBlock {
  int r0, r1, c0, c1;   // rows r0..r1-1, columns c0..c1-1 (0-based: row m = r0+1, ...)
  int k;                // rank
  std::vector<double> U;  // (r1-r0) x k, row-major
  std::vector<double> V;  // (c1-c0) x k, row-major;  block = U V^T
};

struct DenseBlock {
  int bi, bj;               // leaf-row / leaf-column index
  std::vector<double> D;    // L x L row-major
};

struct HostH {
  double alpha = 0, gamma = 0, T = 0;
  int M = 0, L = 0, nb = 0;
  int rank = 0;             // > 0: fixed Taylor terms, no recompression
  double tol = 0;           // > 0: recompression tolerance (block-relative)
  bool dense_mode = false;  // rank == 0 && tol == 0: every lower block dense
  std::vector<double> t;    // mesh, M+1
  std::vector<double> dmm;  // initial-data weights d_{m,m}, M
  std::vector<DenseBlock> dense;  // includes the diagonal blocks
  std::vector<int> diag;          // per leaf row: index into dense
  std::vector<RkBlock> rk;
  int max_rank = 0;
  int taylor_terms = 0;
};

// Flattened, leaf-row ordered form used by the kernels (all offsets in elements).
struct FlatH {
  int M, L, nb;
  int pool_rows;                    // z-pool rows needed (max live sum of ranks)
  // dense off-diagonal blocks per leaf row (j < i), then diagonal handled separately
  std::vector<int> dptr;            // nb+1: range into dlist
  std::vector<int> dlist_blk;       // index into dense block storage
  std::vector<int> dlist_col;       // leaf-column index j
  std::vector<double> dense_data;   // nd x L x L
  std::vector<int> diag_blk;        // nb: block index of the diagonal block
  // U panels: leaf row i uses rows iL..iL+L-1 of every Rk block covering it
  std::vector<int> uptr;            // nb+1: range of panel columns (z rows) per leaf row
  std::vector<int> uz;              // z-pool row of each panel column
  std::vector<long long> uoff;      // nb: element offset of the L x K_i panel (row-major)
  std::vector<double> udata;
  // V panels: leaf row i contributes V^T x_i to every Rk block whose columns cover it
  std::vector<int> vptr;            // nb+1
  std::vector<int> vz;              // z-pool row written by each panel row
  std::vector<int> vinit;           // 1: first leaf of the block's columns (assign, not add)
  std::vector<long long> voff;      // nb: element offset of the K'_i x L panel (row-major)
  std::vector<double> vdata;
  long long flops_per_col_matvec;   // 2 * (stored lower entries touched) per column, matvec
  long long flops_per_col_solve;
};

// The H-matrix as a stream of chunks that the panel kernel stages into shared memory, one
// chunk per pipeline slot, in the order a leaf-row walk consumes them.  Every chunk matrix is a
// product operand out[r] += sum_k A(k, r) in[k] stored vector-interleaved: with VE = 16 / elem
// bytes, entry (k, r) of an R-row matrix sits at ((k / VE) * R + r) * VE + k % VE, so that one
// thread reads VE consecutive k of its row as one 16-byte load and consecutive rows are
// consecutive vectors.  Per leaf row i:
//   DENSE(j)  one L x L near-field block D_ij (k = column, r = row)        (aux = j)
//   UPART     count <= L columns of the U panel (k = panel column, r = row; count padded to whole
//             vectors with zero columns), then count z-pool rows (int)
//   DIAG      D_ii (the smoother streams its level inverse instead; FP32 streams carry both
//             without their diagonal, which the kernels apply in FP64)     (aux = i)
//   VPART     count <= L rows of the V panel (r = panel row, k = column), then one int per row:
//             2 * z-pool row + 1 if the row starts its block's z (assign, not add)
// Chunk descriptor (4 ints): type | count << 4 | (last chunk of its leaf row) << 12, aux, bytes,
// byte offset / 16.  Every chunk
// starts on a 16-byte boundary and its size is a multiple of 16 bytes (TMA bulk copy rule).
enum ChunkType { CH_DENSE = 0, CH_UPART = 1, CH_DIAG = 2, CH_VPART = 3 };

// Writes the row-major L x L matrix A in the chunk layout above (R = L, k = column), optionally
// without its diagonal: the layout of the level inverses the smoother streams as DIAG chunks.
void to_panel_layout(const double* A, int L, int elem_bytes, bool zero_diag, double* out);

struct PanelHost {
  std::vector<unsigned char> pkg;
  std::vector<int> chunks;   // 4 ints per chunk
  std::vector<int> cptr;     // nb+1 chunk ranges per leaf row
  int slot_bytes = 0;        // largest chunk
  int W = 1;                 // depth of the ring of x tiles (max near-field distance + 1, <= 8)
  bool far = false;          // some near-field block lies further back than the ring reaches
};

// elem_bytes = 8 (FP64 matrices) or 4 (FP32 matrices)
void build_panel(const HostH& h, const FlatH& f, int elem_bytes, PanelHost& out);

// The same stream for the tensor-core walk (FP32 products as three TF32 products, hi*hi + hi*lo +
// lo*hi): every chunk matrix (R rows, K reduction index) is padded with zeros to multiples of 16
// and stored as TF32 pairs hi = tf32(a), lo = tf32(a - hi) in the order in which the mma.sync
// m16n8k8 A operand is loaded, one 16-byte vector per lane: float index
//   ((((rt * NKB + kb) * 2 + hl) * 2 + half) * 32 + lane) * 4 + e
// holds part hl (0 hi, 1 lo) of entry (rt*16 + half*8 + lane/4, kb*16 + 4*(lane%4) + e), NKB = K/16.
// A warp's load of one (rt, kb, hl, half) is 512 contiguous bytes.  DENSE and DIAG: R = K = L;
// UPART: R = L, K = count padded to 16 (z indices padded with the slab's first); VPART: R = count
// padded to 16, K = L.  The DIAG blocks carry no diagonal (applied in the grid precision).
void build_panel_mma(const HostH& h, const FlatH& f, PanelHost& out);
// The row-major L x L matrix A in that layout (hi/lo pairs, L*L*2 floats for L a multiple of 16).
void to_mma_layout(const double* A, int L, bool zero_diag, float* out);

// The same stream for FP64-accurate products in double-float arithmetic (pairs of floats, hi =
// fl32(a), lo = fl32(a - hi), |a - hi - lo| <= 2^-48 |a|): the FP32 vector-interleaved layout of the
// hi parts of a chunk matrix (R x K, K padded to a multiple of 4), then the lo parts in the same
// layout, then the chunk's int indices.  DIAG blocks keep their diagonal (products only).
void build_panel_df(const HostH& h, const FlatH& f, PanelHost& out);


// The same stream for the tcgen05 walk (BF16 products, FP32 accumulation in tensor memory): every
// chunk matrix is the B operand of tcgen05.mma kind::f16, R rows (the outputs) by K (the reduction
// index), K-major in the canonical layout without swizzle: 8 x 8 core matrices of 128 contiguous
// bytes (row-major, 16 bytes per row), entry (r, k) at byte umma_offset(r, k, K) =
// ((r/8) (K/8) + k/8) 128 + (r%8) 16 + (k%8) 2, so that adjacent core matrices along K are 128 bytes
// apart (the descriptor's leading byte offset) and adjacent row groups (K/8) 128 bytes apart (its
// stride byte offset).  DENSE: R = K = L; UPART: R = L, K = count padded to 16 (padding columns zero,
// their z indices the slab's first), then the K z indices; DIAG: D_ii without its diagonal (applied
// in FP32 by the kernel); VPART: R = count padded to 16 (zero rows), K = L, then count codes.
void build_panel_umma(const HostH& h, const FlatH& f, PanelHost& out);
size_t umma_offset(int r, int k, int K);
// The row-major L x L matrix A in that layout (BF16 bits, L*L values), optionally without its diagonal.
void to_umma_layout(const double* A, int L, bool zero_diag, uint16_t* out);

// Digit tiles of the tensor-core defect (split.cuh) from the dense time matrix R (row-major M x M,
// lower triangular, M a multiple of 128).  Row m gets the exponent E_m = frexp exponent of
// max_k |R_mk| (so max_k |R_mk| < 2^E_m; 0 for a zero row); R_mk 2^{49 - E_m} rounded to an
// integer X is split into 7 balanced base-2^7 digits, X = sum_a d_a 2^{7 (6 - a)} (|d_0| <= 129,
// the others in [-64, 64]), from the least significant up.  For every output block I (rows
// 128 I ..) and K-block J <= 2 I + 1 (columns 64 J ..), I-major, the digit tiles a whose entries are
// not all zero are stored in ascending a, each 128 x 64 BF16, K-major with the 128-byte swizzle
// (row r's 16-byte chunk c at (r / 8) 1024 + (r % 8) 128 + (c ^ (r % 8)) 16);
// pairs holds {mask of the stored digits, index of the first stored tile, 0, 0} per (I, J).
struct SplitHost {
  std::vector<uint16_t> tiles;
  std::vector<int> pairs;
  std::vector<int> rexp;
};
void build_split(const std::vector<double>& R, int M, SplitHost& out);

// Two-grid convergence factor by mode analysis (sama.cpp): the largest spectral radius of the
// per-mode-group two-grid matrices with the time matrix replaced by its diagonal entries rdiag.
double sama_two_grid(const std::vector<double>& rdiag, int dim, int N, double h, int nu1, int nu2);

// Builds the H-matrix (or the dense lower-triangular R when rank == 0 && tol == 0).  lowrank 0:
// admissible blocks from the Taylor expansion of the kernel (Section 3); 1 (needs rank == 0, tol > 0):
// built algebraically from single entries by adaptive cross approximation, then recompressed.
// Returns 0 on success, < 0 on invalid arguments.
int build_hmatrix(double alpha, double gamma, double T, int M, int leaf, int rank, double tol,
                  HostH& out, int lowrank = 0);
void flatten(const HostH& h, FlatH& f);

// Accurate single entry R_{m,j} (1-based, 1 <= j <= m), used for dense blocks.
double l1_entry(const std::vector<double>& t, double alpha, int m, int j);

// (D_ii + s I)^{-1} for every diagonal leaf block (lower-triangular L x L, row-major).
void diag_inverses(const HostH& h, const FlatH& f, double shift, std::vector<double>& out);

}  // namespace fhmg

// Host-side declarations shared by the translation units of libmsc.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace msc {

enum { PREC_F64 = 0, PREC_F32 = 1 };
enum { OP_STAGGERED = 0, OP_BSR = 1 };
// operator pass kinds
enum {
    PASS_A = 0,  // out = D src (staggered) | out = (A+d) src (BSR); reduce P terms
    PASS_B = 1,  // staggered: r -= alpha (d aux - D src); reduce |r|^2
    PASS_C = 2,  // out = b - (d aux - D src) | b - (A+d) src; reduce |out|^2
    PASS_D = 3,  // out = d aux - D src | (A+d) src
    PASS_BC = 4, // PASS_B inside a conditional chunk graph (sets the update condition)
};

struct StagGeom {
    int L[4];
    int V;
    // 0: the operator on the whole lattice. 1 + p: the parity-reduced
    // operator m^2 - D_{p,1-p} D_{1-p,p} of a source on the sites of parity
    // p = (x0 + x1 + x2 + x3) mod 2; its vectors hold those sites only, in
    // site order (compressed index x / 2), and D passes alternate parities.
    int eo = 0;
    // Division by the divisors d_k = L0, L1, L2, L0 / 2 as a multiply-high
    // (Granlund and Montgomery, "Division by invariant integers using
    // multiplication", 1994): x / d_k = (umulhi(x, dm[k]) + x) >> ds[k] for
    // 0 <= x < 2^31, with ds = ceil(log2 d) and dm = floor(2^(32+ds) / d) + 1
    // - 2^32. Set by stag_geom().
    unsigned dm[4];
    int ds[4];
};
// sites a vector of the operator holds
__host__ __device__ __forceinline__ int vlen(const StagGeom& g) { return g.eo ? (g.V >> 1) : g.V; }
// x / d_k (see StagGeom::dm) for 0 <= x < 2^31
__device__ __forceinline__ int gdiv(int x, const StagGeom& g, int k) {
    return (int)((__umulhi((unsigned)x, g.dm[k]) + (unsigned)x) >> g.ds[k]);
}
// The geometry of a lattice of extents dims[0..3] (each >= 2, V < 2^31).
StagGeom stag_geom(const int dims[4]);

// Device-resident operator data.
struct OpDev {
    int kind;
    int64_t n;  // complex unknowns
    // staggered
    int nc;
    StagGeom g;
    double mass;
    int recon;          // FP32 links keep nc-1 rows
    double2* links64;   // [4][nc*nc][V]
    void* links32;      // full: float2 [4][nc*nc][V]; recon: float4 [4][k][V]
    // block-CSR in sliced-ELL form, 32 rows per slice
    int bd;
    int64_t nbr, nslices, nslots_blk;
    int32_t* slice_len;
    int64_t* slice_start;
    int32_t* cols;      // [slot][32]
    double2* vals64;    // [slot][bd*bd][32]
    float2* vals32;
};

// kernel launchers (return the launch error)
// `act` (device, optional): {count, indices} of the passes to run (see
// sys_block in common.cuh); null runs all npass.
// per_system: one whole grid row per pass (see sys_block).
cudaError_t launch_stag_pass(const OpDev& op, int prec, int kind, int out_f32, const Engine& e,
                             const PassDesc* d_descs, int npass, cudaStream_t st, const int* act = nullptr,
                             bool per_system = false);
// FP32 staggered passes of several systems sharing the operator, the links
// loaded once per group of systems (PASS_A and PASS_B of a solve stage;
// every descriptor has a reduction row; FP32 vectors colour-planar). `act`
// as above. stag_group_applies() says whether a pass takes this path.
bool stag_group_applies(const OpDev& op, int prec, int kind, int npass);
int stag_group_shape();
cudaError_t launch_stag_group(const OpDev& op, int kind, const Engine& e, const PassDesc* d_descs, int npass,
                              cudaStream_t st, const int* act);
// One FP32 system (PASS_A, PASS_B) with the links of each tile of sites
// staged in shared memory by bulk asynchronous copies; stag_tile_fits() says
// whether the lattice can be cut into such tiles (recon links only). A wait
// on the copies that runs out after wait_ns sets bit 0 of *e.err; no_copy
// issues none (a test of that path).
bool stag_tile_fits(const StagGeom& g, int nc);
size_t stag_tile_smem(int nc, int L0);
cudaError_t launch_stag_tile(const OpDev& op, int kind, const Engine& e, const PassDesc* d_descs, uint64_t wait_ns,
                             int no_copy, cudaStream_t st);
// h_desc (optional): host copy of the single pass's descriptor; a one-system
// FP32 PASS_A then takes its source and output pointers from it as kernel
// parameters (the device descriptor must hold the same pointers).
cudaError_t launch_bsr_pass(const OpDev& op, int prec, int kind, int out_f32, const Engine& e,
                            const PassDesc* d_descs, int npass, cudaStream_t st, const int* act = nullptr,
                            bool per_system = false, const PassDesc* h_desc = nullptr);
// FP32 SpMV of several systems sharing the matrix, `group` (1 or 2)
// systems per block row of the grid, `groups` rows; `act` (device, optional)
// = {count, indices...} of the systems to run, read when the kernel runs.
// kMultiGroup: the group size the solver uses for two or more systems.
constexpr int kMultiGroup = 2;
cudaError_t launch_bsr_multi(const OpDev& op, const Engine& e, const PassDesc* d_descs, int npass,
                             const int* act, int group, int groups, cudaStream_t st);

// vector kernels; vectors are addressed as [index][npad] complex in the
// iteration precision (prec) unless noted
struct VecSet {
    void* r;        // [nsys][npad]
    void* p;        // [nsys][npad]
    void* t;        // [nsys][npad] (t = D p or Ap)
    void* ps;       // [slots][npad]
    void* xit;      // [slots][npad] x accumulator in iteration precision
    double2* x64;   // [slots][npad]
    const double2* b64;  // [rhs][npad]
    int64_t npad;
    // pl_nc > 0: the iteration-precision (FP32) vectors are colour-planar,
    // entry (site x, colour a) at a * pl_V + x (staggered operators); the
    // FP64 vectors stay site-major (x * pl_nc + a). 0: all site-major.
    int pl_nc = 0;
    int pl_V = 0;
};
cudaError_t launch_init(int prec, const Engine& e, const VecSet& v, const PassDesc* d_descs,
                        int nsys, cudaStream_t st);
cudaError_t launch_init_from_r(int prec, const Engine& e, const VecSet& v, int nsys, cudaStream_t st);
cudaError_t launch_update(int prec, const Engine& e, const VecSet& v, int nsys, cudaStream_t st,
                          const int* act = nullptr);
cudaError_t launch_axpy_norm(int prec, const Engine& e, const VecSet& v, const PassDesc* d_descs,
                             int nsys, cudaStream_t st, const int* act = nullptr);
cudaError_t launch_fold(const Engine& e, const VecSet& v, int nsys, int only_ru, cudaStream_t st,
                        const int* act = nullptr, bool per_system = false);
cudaError_t launch_convert(const void* src, int src_f32, void* dst, int dst_f32, int64_t n,
                           cudaStream_t st);
// FP64 site-major <-> FP32 colour-planar copy of one vector of V sites x nc
// colours (to_planar: src FP64, dst FP32; else the reverse).
cudaError_t launch_convert_planar(const void* src, void* dst, int nc, int V, bool to_planar, cudaStream_t st);

// right-hand sides of polynomial form (FP64, [s][npad] site-major vectors,
// one launch for all S shifts): a Horner step v_s = Av_s + a_s b (Av null:
// v_s = a_s b); the solution x_s = c_s x_s + x0_s (x0 null: c_s x_s); and
// e.out_red[s] = |v_s|^2 for s < count (uses reduction rows 0 .. count-1).
struct ShiftCoef {
    double v[kMaxShifts + 1];
};
cudaError_t launch_poly_step(double2* v, const double2* Av, const ShiftCoef& a, const double2* b, int S,
                             int64_t n, int64_t npad, cudaStream_t st);
cudaError_t launch_poly_combine(double2* x, const double2* x0, const ShiftCoef& c, int S, int64_t n, int64_t npad,
                                cudaStream_t st);
cudaError_t launch_norms(const Engine& e, const double2* v, int count, int64_t n, int64_t npad, cudaStream_t st);

// set-up kernels
cudaError_t stag_pack_links(OpDev& op, const double2* links_aos, double* d_maxdev,
                            cudaStream_t st);
cudaError_t stag_unitarity(const OpDev& op, const double2* links_aos, double* d_maxdev,
                           cudaStream_t st);
cudaError_t stag_pack_links32(OpDev& op, const double2* links_aos, cudaStream_t st);
cudaError_t stag_export_bsr(const OpDev& op, int64_t* row_ptr, int32_t* col, double2* vals,
                            cudaStream_t st);
// max |A_ij - conj(A_ji)| and max |A_ij| over the entries of a block-CSR
// matrix (repeated columns summed) into d_out[0], d_out[1] (FP64 bit
// patterns; d_out zeroed by the caller).
cudaError_t bsr_check_hermitian(const int64_t* d_row_ptr, const int32_t* d_col, const double2* d_vals,
                                int64_t nbr, int bd, unsigned long long* d_out, cudaStream_t st);
cudaError_t bsr_pack(OpDev& op, const int64_t* d_row_ptr, const int32_t* d_col,
                     const double2* d_vals, int* d_bad, cudaStream_t st);

// ---------------------------------------------------------------------------
// batched uneven systems (batch.cu): many staggered operators, one launch per
// pass. Blocks are flattened over systems: block b serves system j with
// map[j] <= b < map[j+1] (separate maps for site and vector kernels).
// ---------------------------------------------------------------------------
struct BOp {             // one staggered operator of a batch
    StagGeom g;
    int nc, recon;
    const void* l32;
    const double2* l64;
};
struct BSys {            // one system of a batch: a right-hand side (or a refined shift)
    int64_t voff;        // offset (complex) of its r, p, t and t64 rows
    int64_t soff;        // offset (complex) of its first shift slot in x64 / xit / ps
    int64_t boff;        // offset (complex) of its source in b64
    int npad;            // vector length (complex, multiple of 64)
    int op;              // index into the operator table
};
struct BVec {            // base pointers of the batch's vectors
    void* r;
    void* p;
    void* t;
    void* ps;
    void* xit;           // FP32 x accumulators (mixed) or the FP64 x (FP64)
    double2* x64;
    double2* t64;
    const double2* b64;
};
struct BTab {             // device tables of a batched stage
    const BSys* sys;     // [systems]
    const BOp* ops;      // [operators]
    const int* hdr;      // {active systems, site, vector, update virtual blocks}
    const int* act;      // [active] system indices
    const int* msite;    // [active + 1] prefix sums of blocks: operator passes
    const int* mvec;     // [active + 1] one unit per thread (init, fold)
    const int* mupd;     // [active + 1] `units` units per thread (update)
};
cudaError_t launch_b_stag(int prec, int kind, int out_f32, const Engine& e, const PassDesc* descs,
                          const BTab& t, int threads, cudaStream_t st);
cudaError_t launch_b_init(int prec, const Engine& e, const BVec& v, const BTab& t, int threads,
                          cudaStream_t st);
cudaError_t launch_b_init_from_r(int prec, const Engine& e, const BVec& v, const BTab& t, int threads,
                                 cudaStream_t st);
cudaError_t launch_b_update(int prec, int units, const Engine& e, const BVec& v, const BTab& t, int threads,
                            cudaStream_t st);
cudaError_t launch_b_fold(const Engine& e, const BVec& v, const BTab& t, int threads, int only_ru,
                          cudaStream_t st);

// adjoint (force.cu)
cudaError_t launch_quad(const Engine& e, const double2* phi, const double2* x, const double* c, int S,
                        int64_t n, int64_t npad, int row, cudaStream_t st);
cudaError_t launch_dphi(const double2* x, const double* c, int S, int64_t n, int64_t npad,
                        double2* out, cudaStream_t st);
cudaError_t launch_force(const OpDev& op, const double2* x, const double2* y, const double* c, int S,
                         int64_t npad, double2* G, cudaStream_t st);

int grid_blocks(int64_t work, int num_sms);

// Blocks of kThreads for `work` items: one item per thread, capped at the
// blocks that fit on the device at once for kernel `fn` (no partial waves).
int resident_grid(const void* fn, int64_t work);
// Blocks of `threads` threads resident on the device for kernel `fn`
// (occupancy x SMs), at most kMaxBlocks.
int resident_blocks(const void* fn, int threads);
// Grid for `nsys` systems of `work` items each (see sys_block): 1-D, the
// resident blocks and at least one per system; or, per_system, a full row
// of resident blocks for every system.
dim3 multi_grid(const void* fn, int64_t work, int nsys, bool per_system = false);

}  // namespace msc

// Internal interface between the C-ABI host layer (lbm_api.cu) and the kernels
// (lbm_kernels.cuh, instantiated in lbm_f64.cu and lbm_f32.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lbm {

// Node-type bits of the uint8 mask.
constexpr uint8_t kSolid = 1;     // inside the cylinder
constexpr uint8_t kNearWall = 2;  // fluid node with a D2Q9 neighbour inside the cylinder
constexpr uint8_t kNear2 = 4;     // fluid node with a solid node at most 2 nodes away in x and y

// Lattice geometry.  Arrays are [ny][pitch], pitch >= nx a multiple of 32 elements.
struct Geo {
  int nx, ny, pitch, periodic_x;
  int plane;        // elements per population plane = ny * pitch (9 * plane < 2^31)
  double xc, yc, r; // cylinder centre and radius (r <= 0: none)
  // link fractions of the near-wall nodes, tabulated on the host: wall_idx[y * pitch + x] is
  // the node's row (-1 away from the wall); wall_q[row * 8 + i - 1] (compute type) is the
  // fraction of the link from the node along -c_i that lies in the fluid, -1 where the pull
  // source of direction i is fluid
  const int* wall_idx;
  const void* wall_q;
  const double* wall_n;  // [row][2]: outward unit normal (from the centre) of the near-wall node
};

// A double-float value hi + lo (two FP32 words, |lo| <= ulp(hi)/2).
struct F2 {
  float hi, lo;
};

// Physical constants in one precision.
template <typename C>
struct PhysC {
  C a, b, R, kappa, Tc, G, sigma;
  C T_sat, T_wall;
  C rho_l, rho_v, rho_s;
  C nu_l, nu_v, alpha_l, alpha_v, c_v;
  C g, u_in, U_out;
  C U_k;      // U_out / (1 + U_out): the convective outlet's relaxation factor
  C body_fx;  // uniform body force along +x (0: none)
};

// Physical constants, derived on the host in double and rounded once to float there, so
// that no kernel converts a double to a float (on GB300 that conversion runs on the FP64
// pipe).  The double-float copies serve the FP32 build's psi: a, b, R, kappa, 1/Tc,
// cs^2 = 1/3 and k = 2/(G cs^2).
struct Phys {
  PhysC<double> d;
  PhysC<float> f;
  F2 a2, b2, R2, kappa2, invTc2, cs22, k2;
  F2 kR2, ka2, k32;  // k R, k a, k / 3 with k = 2 / (G cs^2): the double-float psi's folded constants
  F2 K12;            // 1 + kappa (the same)
  float dpdT_c1, dpdT_c2;  // kappa (1 + kappa) and kappa^2 / Tc: (dp/dT)_rho of the FP32 energy pass
  float pop_shift[9];  // shifted FP16 storage keeps f_i - w_i rho_l; these are w_i rho_l
};

// psi evaluation of the FP32 build (Eq. potential with Eq. eos); values of lbm_params.psi_mode.
enum PsiMode { kPsiDF = 0, kPsiF64 = 1, kPsiF32 = 2 };
// Launch flags of the single-domain collision and energy passes: bit 0 stage interior tiles by
// TMA; bit 1 (test hook) arm each staged tile's barrier without issuing its copies and wait a
// short bound, so that the bounded wait runs out with nothing in flight.
constexpr int kLaunchStaged = 1, kLaunchStarve = 2;
// The collision may copy its populations before the previous kernel in the stream has ended
// (that kernel is the energy pass of the step before, which does not write them).
constexpr int kLaunchEarlyF = 4;
// Which pass lbm_inject_fault starves; latched status bits of a wait that ran out, per pass.
constexpr int kStarveCollide = 1, kStarveEnergy = 2;
constexpr int kStatusTimeoutCollide = 4, kStatusTimeoutEnergy = 8;
// Collision operator (the values of lbm_collision): the CM collision of Sec. II.A, or the
// single-rate BGK operator of the Sec. III.B comparison.
enum CollisionOp { kCollCM = 0, kCollBGK = 1 };

// Device buffers of one context (type-erased; element type is the storage / compute type).
struct Dev {
  void* f[2];        // populations, 9 planes each (ping-pong)
  void* T[2];        // temperature (ping-pong)
  void* psi;         // pseudopotential of the current step
  void* psi_next;    // pseudopotential of the next step, when the energy pass computed it
  void* t1_out;      // if set, the energy pass also stores its stage-1 temperature T1 here
  void* rho;         // density of the last collision
  void* ux;          // velocity of the last collision
  void* uy;
  void* side[2];     // [3][ny] last streamed f_2, f_6, f_8 at the outlet column (ping-pong with f)
  const uint8_t* mask;
  const int* bnode;  // boundary fluid nodes (y * pitch + x)
  const double* bn;  // their outward normals, [2][nb]
  int nb;
  int tma;           // 1: interior collision tiles are staged by TMA (environment LBM_TMA=0 turns it off)
  int starve;        // test hook for the bounded waits (lbm_inject_fault): kStarve* bits of the next step
  int pdl;           // 1: the step's passes are launched as programmatic dependents of the kernel
                     // before them (environment LBM_PDL=0 turns it off)
  int f_ready;       // 1: this step's populations were written before the kernel preceding its
                     // collision (set by lbm_step for all but the first step of a call)
  int collision;     // LBM_COLL_CM or LBM_COLL_BGK
  double* hf;        // heat-flux accumulators: last, sum, sum of squares, count
  double* partial;   // one heat-flux partial sum per energy-kernel block (zero between launches)
  int wall_tiles[2]; // energy tiles (32 wide, 8 or 16 high) that hold a near-wall node
  unsigned* counter; // blocks of the current energy launch that have finished (wraps to 0)
  int* status;       // latched fault bits
  double* stage;     // nx*ny doubles for exports/imports
};

// One domain of a batch, as the batched kernels see it.  Tiles of every pass are numbered
// consecutively over the domains; *_first is this domain's first tile of that pass.
// Tensor maps of the energy pass's inputs with the box of a tile and its 4-node halo: T, and
// rho, u_x, u_y as three consecutive planes (one 3D box); interior tiles copy them into shared
// memory with TMA.
struct EnergyMaps {
  CUtensorMap T, ruv;
};

struct BatchDomain {
  Geo g;
  Phys ph;
  Dev d;
  long long warmup;
  int energy;
  int psi_first, psi_ntx;                 // psi pass: 32 x 8 tiles
  int coll_first, coll_ntx;               // collision pass: 32 x CTY tiles
  int en_first, en_ntx, en_nblocks;       // energy pass: 32 x ETY tiles
  int tma;                                // 1: the launch passes this domain's tensor maps
};

// Tensor maps of one batched domain for the current tile variant (kept on the host): the
// populations and psi of population parity 0 / 1 for the collision pass, and the energy
// inputs with T of parity 0 / 1.  A batched launch passes the current parity's maps of a
// range of domains as kernel parameters (at most about 32 KB of them), hence the ranges below.
struct DomainMaps {
  CUtensorMap f[2], psi[2];
  EnergyMaps em[2];
};
constexpr int kBatchCollDomains = 126, kBatchEnDomains = 126;
struct CollLaunchMaps {
  CUtensorMap f[kBatchCollDomains], psi[kBatchCollDomains];
};
struct EnLaunchMaps {
  EnergyMaps e[kBatchEnDomains];
};

// Encode the tensor maps of one batched domain for tile heights (cty, ety); sets D.tma to
// whether all of them could be made.
bool batch_maps_f32(BatchDomain& D, DomainMaps& m, int cty, int ety);
bool batch_maps_f64(BatchDomain& D, DomainMaps& m, int cty, int ety);

// Tile-height variants of the batched step the autotuner chooses from: (CTY, ETY).
constexpr int kBatchVariants = 4;
inline void batch_variant(int v, bool f64, int& cty, int& ety) {
  cty = (v & 1) ? 16 : 8;
  ety = f64 ? 8 : ((v & 2) ? 8 : 16);
}

// Batched step over all domains (one launch per pass).  maps: block -> domain index for
// the psi, collision and energy passes; need_psi: run the psi pass first (psi of the current
// state is not known from the last energy pass).  Returns the number of launches or -1.
// hdoms, hmaps, ndom: the host copies of the domains (their first tiles) and their tensor maps.
int batch_step_f32(int variant, const BatchDomain* doms, const int* map_psi, int nb_psi, const int* map_coll,
                   int nb_coll, const int* map_en, int nb_en, int cur, int tcur, long long step, int need_psi,
                   const BatchDomain* hdoms, const DomainMaps* hmaps, int ndom, cudaStream_t s);
int batch_step_f64(int variant, const BatchDomain* doms, const int* map_psi, int nb_psi, const int* map_coll,
                   int nb_coll, const int* map_en, int nb_en, int cur, int tcur, long long step, int need_psi,
                   const BatchDomain* hdoms, const DomainMaps* hmaps, int ndom, cudaStream_t s);

// Kernel identifiers for per-launch timing.
enum KernelId { kKRhoPsi = 0, kKCollide, kKEnergy, kKExport, kKImport, kNumKernels };

// Tile shapes (threads per block = tile nodes).
constexpr int kEnergyTX = 32, kEnergyTY = 16;
inline int energy_blocks(int nx, int ny) {  // upper bound over both precisions (FP64 tiles are 32x8)
  return ((nx + kEnergyTX - 1) / kEnergyTX) * ((ny + 7) / 8);
}
extern const char* const kKernelNames[kNumKernels];

// Per-launch hook: called before and after each kernel launch of a step.
struct LaunchHook {
  void (*before)(void* self, int kernel);
  void (*after)(void* self, int kernel);
  void* self;
};

// psi of the next step from the energy pass: have = d.psi already holds psi of this step (no
// psi pass), want = the energy pass should write psi of the next step into d.psi_next; made is
// set when it did.
struct PsiChain {
  int have, want, made;
};

// Step launchers (one per precision build).  cur: index of the buffers holding f* and the
// outlet side values; tcur: index of the temperature buffer.  The step writes f*, side into
// [cur ^ 1] and, when it runs the energy equation, T into [tcur ^ 1] (*t_flipped = 1).
// Returns the number of kernels launched, or -1 on a launch error.
int step_f64(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int forcing, int energy, int psi_mode,
             cudaStream_t s, const LaunchHook* hook, int* t_flipped, PsiChain* chain = nullptr);
// FP32 compute with population storage `storage` (lbm_storage: 0 FP64, 1 FP32, 2 shifted FP16).
int step_f32(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int forcing, int energy, int psi_mode,
             int storage, cudaStream_t s, const LaunchHook* hook, int* t_flipped, PsiChain* chain = nullptr);

// Field export: copy a typed [ny][pitch] field (which: 0 rho, 1 ux, 2 uy, 3 T, 4 psi, 5 solid,
// 10+i population plane i of buffer cur, 20+j outlet side row j of buffer cur, 30 + comp + 2 *
// forcing the force component comp of the last collision) into a dense double buffer.  T is
// taken from buffer tcur.
int export_f64(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int which, double* dst, cudaStream_t s);
int export_f32(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int which, int storage, double* dst,
               cudaStream_t s);
// Field import: the reverse, for T (3), population planes (10+i) and side rows (20+j).
int import_f64(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int which, const double* src,
               cudaStream_t s);
int import_f32(const Geo& g, const Phys& ph, const Dev& d, int cur, int tcur, int which, int storage,
               const double* src, cudaStream_t s);
// Initial state: populations at the Hermite equilibrium of (rho0 + drho, ux0, uy0), T = T0;
// array arguments are dense [ny][nx] device doubles or NULL (see lbm_init in lbm.h).
// Tw: dense wall temperatures of the solid nodes (NULL: T_wall everywhere).
int init_f64(const Geo& g, const Phys& ph, const Dev& d, const double* rho0, const double* drho, const double* ux0,
             const double* uy0, const double* T0, const double* Tw, unsigned long long seed, double amp,
             cudaStream_t s);
int init_f32(const Geo& g, const Phys& ph, const Dev& d, const double* rho0, const double* drho, const double* ux0,
             const double* uy0, const double* T0, const double* Tw, unsigned long long seed, double amp, int storage,
             cudaStream_t s);

// Arguments of the reverse step (lbm_adjoint.cuh): typed [ny][pitch] planes of one context.
template <typename C>
struct AdjArgs {
  Geo g;
  Phys ph;
  const uint8_t* mask;
  // forward: state entering the step and the fields of its collision
  const C* f;     // f* (9 planes)
  const C* T;
  const C* side;  // [3][ny]
  const C* rho;
  const C* psi;
  const C* ux;
  const C* uy;
  const C* T1;    // the step's stage-1 temperature (stored by its recompute)
  // adjoint seeds on the step's outputs, and the results on its inputs
  const C* fb_in;
  const C* Tb_in;
  const C* sb_in;
  C* fb_out;
  C* Tb_out;
  C* sb_out;
  // work planes
  C* Tb1;         // adjoint of the stage-1 temperature
  C* ub[2];       // adjoint of u from the energy equation
  C* lamb;        // adjoint of lambda (stage 2)
  C* rhob;        // adjoint of rho from the energy equation and lambda
  C* fpb;         // adjoint of the pulled populations (9 planes)
  C* fmb[2];      // adjoint of the interaction force F_m
  C* psib;        // adjoint of psi from the consistency terms
  double* gw;     // dJ/dT_w per node (solid nodes), accumulated
  double* uin;    // dJ/du_in per inlet row, accumulated
  C wq;           // weight of this step's heat-flux sample in the objective
  int do_hf;
};

// One reverse step of the time step (8 launches); returns the number of launches or -1.
int adjoint_step_f32(const AdjArgs<float>& a, cudaStream_t s);
int adjoint_step_f64(const AdjArgs<double>& a, cudaStream_t s);
// Per-device set-up of the adjoint kernels (shared-memory opt-in); 0 or -1.
int adjoint_setup_f32();
int adjoint_setup_f64();
// Plane helpers of the adjoint: op 0 T[solid] = wallT (src wallT, dst T); op 1 gw[solid] +=
// Tb (src Tb, dst gw doubles); op 2 dense doubles -> typed plane; op 3 typed plane -> dense.
int adjoint_aux_f32(int op, const Geo& g, const uint8_t* mask, const void* src, void* dst, cudaStream_t s);
int adjoint_aux_f64(int op, const Geo& g, const uint8_t* mask, const void* src, void* dst, cudaStream_t s);

}  // namespace lbm

// dot_batch.cuh -- a batch of G mixed-precision solves of one grid (path_mixed.cu).
//
// Every per-solve field is stored as G consecutive copies (MxFields / slot_view),
// the DCT tables are shared, and each launch of Algorithm 2's kernels advances
// every active slot at once.  The penalty of each slot lives in a device array of
// SlotParam, so one captured launch sequence (a CUDA graph) serves every sigma and
// every set of active slots: slots are filled and emptied between launches.
// A single solve (dot_create) is a batch with G = 1.
#pragma once
#include <memory>
#include <string>
#include <vector>

#include "dot_mixed.cuh"
#include "dot_paths.cuh"

namespace dot {

class MixedBatch {
 public:
  MixedBatch(const Geo& g, int G, bool slot_masks);
  ~MixedBatch();
  // Bytes of the workspace for G slots; slot_masks: every slot carries omega
  // arrays (a batch serving masked and unmasked solves together).
  static size_t workspace_bytes(const Geo& g, int G, bool slot_masks);
  // Whether G > 1 slots of this grid can share the launches (the batched Poisson
  // flow needs every axis on the tensor cores).
  static bool batchable(const Geo& g);

  // Carve the workspace, upload the DCT tables, mark every slot empty.
  int init(char* ws, size_t bytes, cudaStream_t s, std::string* err);
  // Put a new solve into slot b: densities (c, scaled as in dot_create), omega
  // (nullptr: 1 everywhere), a zero iterate, the penalty sigma.  Stream-ordered.
  int load_slot(int b, const std::vector<double>& m0, const std::vector<double>& m1,
                const std::vector<double>* omega, double sigma, double tau, cudaStream_t s, std::string* err);
  // Host copy of the slot parameters; upload_params copies them to the device.
  // set_sigma with rescale: the slot's stored multipliers (alpha/sigma, beta/sigma)
  // belong to the old sigma and are rescaled by the next apply_rescale.
  void set_sigma(int b, double sigma, double tau, bool rescale);
  double sigma(int b) const { return hs_[b]; }
  // Rescale the stored multipliers of every slot whose sigma changed (one kernel;
  // it reads the factors from the device parameters), and mark them done on the host.
  void apply_rescale(cudaStream_t s, LaunchCounter lc);
  void clear_rescale();
  bool rescale_pending() const;
  void set_active(int b, bool on);
  bool active(int b) const { return hp_[b].active != 0; }
  cudaError_t upload_params(cudaStream_t s);
  // whether the host parameters changed since the last upload
  bool params_dirty() const { return params_dirty_; }
  // After a check period: clear every slot's assemble flag (the fused kernels left a
  // valid residual for each); a penalty change or a new state sets it again.
  void end_period();

  // One iteration of Algorithm 2 for every active slot.
  void iterate(cudaStream_t s, LaunchCounter lc);
  // Stopping-measure sums of every active slot into red_out()[G][R_NSLOTS].
  void kkt(cudaStream_t s, LaunchCounter lc);
  const double* red_out() const { return red_; }
  const int* error_flag() const { return err_; }
  void set_tensor_cores(bool on) { ps_.use_tc = on; }
  int slots() const { return G_; }
  // Which of the two (q, alpha, beta) sets is current.  A stream capture of
  // iterate() flips it without running anything; set_parity puts it back.
  int parity() const { return cur_; }
  void set_parity(int p) { cur_ = p & 1; }
  // Whether the next iterate() reuses the residual the previous one left in f.r.
  bool residual_valid() const { return r_valid_; }
  const Geo& geo() const { return g_; }

  int read_fields(int b, double* rho, double* m, double* phi, cudaStream_t s, std::string* err);
  int read_state(int b, double* q, double* al, double* beta, cudaStream_t s, std::string* err);
  int write_state(int b, const double* q, const double* al, const double* beta, double sigma, double tau,
                  cudaStream_t s, std::string* err);
  // The refined Poisson operator on slot 0's scratch.
  int poisson_op(const double* b, double* phi, cudaStream_t s, LaunchCounter lc, std::string* err);

  struct Buffers;   // device buffer plan (path_mixed.cu)

 private:
  Geo g_;
  int G_;
  bool slot_masks_;
  bool fused_ = false, tma_ = false, fused3_ = false;
  int cur_ = 0;
  bool r_valid_ = false;   // f.r holds the next iteration's residual (from the fused kernel)
  bool params_dirty_ = true;
  std::unique_ptr<Buffers> B_;
  MxPoisson ps_;
  double* red_ = nullptr;
  int* err_ = nullptr;
  SlotParam* dparams_ = nullptr;
  std::vector<SlotParam> hp_;
  std::vector<double> hs_;   // sigma per slot (host)
  std::vector<std::vector<float>> hT_;

  const MxFields& cur() const;
  const MxFields& other() const;
  cudaError_t zero_slot(int b, cudaStream_t s);
};

}  // namespace dot

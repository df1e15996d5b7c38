// fd_internal.h -- the library's handle types, shared by its translation units.
#pragma once

#include <stdint.h>

#include <vector>

#include "../../include/fd_gb300.h"

struct fd_chain_s {
  int device = 0;
  int32_t n_chains = 0;
  int64_t n_links = 0;
  int32_t max_links = 0;
  double grav[3] = {0, 0, 0};
  std::vector<int64_t> h_off;
  void *d_model64 = nullptr;
  void *d_model32 = nullptr;
  int64_t *d_off = nullptr;
  bool rigid = true;  // every inertia has the rigid-body form (mass gradients)
  int32_t *d_parent = nullptr;  // kinematic trees: [n_links] parent within the tree; null: chains
  std::vector<double> h_axes;   // kinematic trees: the joint axes as given ([n_links][3])
  std::vector<int32_t> h_parent;
  // closed loops (fd_tree_add_loops): per tree a range of loops, per loop links
  // a, b and the two joint frames in canonical link coordinates
  int32_t n_loops = 0;
  int32_t *d_loop_off = nullptr;  // [n_chains + 1]
  int32_t *d_loop_ab = nullptr;   // [n_loops][2]
  double *d_loop_T = nullptr;     // [n_loops][24]
};

struct fd_batch_s {
  fd_chain_t chain = nullptr;
  int device = 0;  // the chain set's device, kept so the plan can be freed on its own
  int32_t n_problems = 0;
  int64_t n_state_links = 0;
  int64_t sum_sq = 0;
  int32_t max_links = 0;
  int32_t *d_prob_chain = nullptr;
  int64_t *d_state_off = nullptr;
  int64_t *d_sq_off = nullptr;
  int32_t *d_order = nullptr;
  int tuned[FD_N_ALGOS][3] = {};  // autotuned team per [algo][prec]
  // Length classes: problems whose link counts share ceil(log2 n) (n <= 1: class
  // 0), as contiguous ranges [first, first + count) of the processing order
  // (longest first). A batch with more than one class is solved with team 0 in
  // one launch whose grid is split by class, each class with its own team.
  struct LenClass {
    int32_t key, first, count, min_len, max_len;
  };
  std::vector<LenClass> classes;
  std::vector<int> ctuned;  // autotuned team per [class][algo][prec] (0: not tuned)
};

// Sets the calling thread's fd_last_error message and returns st.
fd_status fdk_fail(fd_status st, const char *msg);

// The team size used when a caller passes team 0 and nothing was autotuned: a
// size that fills the GPU for n_problems problems of up to max_links links.
int fdk_default_team(int32_t algo, int64_t n_problems, int32_t max_links);

// Team sizes the kernels are built for: powers of two from 1 to 256.
bool fdk_valid_team(int t);

// Packs one chain's (or tree's) model records in canonical link frames (see
// fd_abi.cu). parents: null for a serial chain, else each link's parent within
// its tree (-1: the base), indexed like the other arrays.
fd_status fdk_pack_chain(int64_t first, int64_t n, const double *joint_axes,
                         const double *link_frames, const double *spatial_inertias, double *rec,
                         bool *rigid, const int32_t *parents = nullptr);

"""GB300-native Stop-and-Stare (SSA / D-SSA) influence maximisation.

The compute path is libssa.so (hand-written sm_103a CUDA behind the C ABI in
include/ssa.h); this package only builds it and marshals arguments."""
from .binding import (SSA_ALGO_DSSA, SSA_ALGO_SSA, SSA_IC, SSA_LT, SSA_W_EXPLICIT, SSA_W_TRIVALENCY, SSA_W_WC,
                      EXPORTS, Graph, Pool, Result, Solver, SSAError, lib, ssa_autotune, ssa_set_tuning, ssa_set_wait_polls, ssa_set_queue_tuning, ssa_set_greedy_mode, ssa_set_warp_tier, ssa_set_lane_tier, ssa_coverage, ssa_coverage_noalloc,
                      ssa_estimate_inf, Server, ssa_server_create, ssa_server_destroy, ssa_server_poll,
                      ssa_server_stats, ssa_server_submit, ssa_server_wait,
                      ssa_free_graph, ssa_gen_rmat, ssa_graph_export, ssa_graph_info, ssa_load_graph, ssa_max_coverage,
                      ssa_pool_create, ssa_pool_grow, ssa_solve, ssa_solver_create, ssa_solver_free,
                      ssa_solver_solve, ssa_version, ssa_device_code_version)

__all__ = [n for n in dir() if n.startswith(("ssa_", "SSA_"))] + ["Graph", "Pool", "Result", "Server", "Solver", "SSAError",
                                                                  "EXPORTS", "lib"]

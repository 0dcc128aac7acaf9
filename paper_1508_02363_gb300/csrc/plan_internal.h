// Slot-level interface of a plan, used by the serving runtime (serve.cu):
// slots are loaded, started, advanced one cycle at a time and read back
// independently of each other.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <string>

#include "../../include/dbar.h"

struct dbar_plan;

dbar_status dbar_internal_fail(dbar_status st, const std::string& msg);

// Device bytes one slot costs, and the slot-independent tables of a plan.
size_t plan_slot_bytes(const dbar_params* p, int per_slot_q);
size_t plan_fixed_bytes(const dbar_params* p);
// per_slot_q = 1: each slot has its own potential Q (loaded by plan_load_slot).
dbar_status plan_create_ex(const dbar_params* p, int per_slot_q, dbar_plan** out);
int plan_batch(const dbar_plan* P);
size_t plan_device_bytes(const dbar_plan* P);
// Copies Q (host, N*N complex128, physical layout) and E_k for k = k1 + i k2 into slot.
dbar_status plan_load_slot(dbar_plan* P, int slot, const double* Q, double k1, double k2, cudaStream_t st);
// Starts the slots with hmask[s] != 0 (x = 0, right-hand side, first cycle state).
dbar_status plan_begin(dbar_plan* P, int nb, const int* hmask, cudaStream_t st);
// Synchronises the stream and returns each slot's "still iterating" flag.
dbar_status plan_active(dbar_plan* P, int nb, int* active, cudaStream_t st);
// One cycle for every active slot among the first nb, in plan_cycle_parts(P) + 1
// parts, one per call, without host synchronisation: part c < plan_cycle_parts(P)
// launches a chunk of Krylov steps and queues a copy of the run flags; once the stream
// has passed it, plan_parts_running says whether any slot still iterates (if none, the
// caller launches the tail part, plan_cycle_parts(P), at once instead of the remaining
// chunks).
int plan_cycle_parts(const dbar_plan* P);
dbar_status plan_step_part(dbar_plan* P, int nb, int part, cudaStream_t st);
bool plan_parts_running(const dbar_plan* P, int nb);
// Reads a finished slot: S (host, N*N complex128), m (nullable), iterations,
// cycles and the final relative residual.  Synchronises the stream.
dbar_status plan_read_slot(dbar_plan* P, int slot, double* S, double* m, int* itot, int* ncyc, double* resid,
                           cudaStream_t st);

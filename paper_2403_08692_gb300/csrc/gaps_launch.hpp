// Host-side launchers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include "gaps_device.cuh"

namespace gaps {

// Launch parameters of a job whose batch event ev has Philox event id
// ev + id_offset.
DevParams make_dev_params(const gaps_params& p, int64_t id_offset);
// Remember a CUDA error for gaps_last_cuda_error() and return GAPS_ERR_CUDA.
int record_cuda_error(cudaError_t e);
Events make_events(const gaps_batch& b);

cudaError_t launch_me(const DevParams& P, const Events& E, cudaStream_t s);
// One plain-form cycle over list_in[0 .. n_in) (list_in = NULL: events
// 0 .. n_in); survivors are appended to list_out (may be NULL) through
// *out_count; *reset_count is zeroed.
// n_in_dev (may be NULL): the list length on the device, n_in then only
// bounds it.
cudaError_t launch_step_plain(const DevParams& P, const Events& E, const int* list_in, int64_t n_in,
                              const unsigned long long* n_in_dev, int* list_out, unsigned long long* out_count,
                              unsigned long long* reset_count, cudaStream_t s);
// One plain-form step with deferred emissions: the select/veto phase for
// list_in[0 .. n_list) (list_in = NULL: events 0 .. n_list) and the
// emissions tasks_in[0 .. n_tasks) accepted by the previous step.  Vetoed and
// emitted events go to list_out, accepted ones to tasks_out; *reset_list and
// *reset_tasks are zeroed.  n_list_dev / n_tasks_dev (may be NULL): the
// lengths on the device, the host ones then only bound them.  With
// *emit_cursor hands out the emission tasks in chunks (zero before the
// launch); *reset_cursor, the next launch's cursor, is zeroed.  With
// pub.slot set (host-mapped memory), the launch writes its input lengths --
// the previous launch's output lengths -- to pub.slot[0..1] as it starts,
// then pub.seq to pub.slot[2], so that the host learns them without a copy
// on the stream.
struct StepPublish {
  unsigned long long* slot;
  unsigned long long seq;
};
cudaError_t launch_step_deferred(const DevParams& P, const Events& E, const int* list_in, int64_t n_list,
                                 const unsigned long long* n_list_dev, const EmitTask* tasks_in, int64_t n_tasks,
                                 const unsigned long long* n_tasks_dev, int* list_out, unsigned long long* list_count,
                                 EmitTask* tasks_out, unsigned long long* task_count, unsigned long long* reset_list,
                                 unsigned long long* reset_tasks, unsigned long long* emit_cursor,
                                 unsigned long long* reset_cursor, StepPublish pub, cudaStream_t s);
// The active list of a batch rebuilt in event order (events with status
// GAPS_ACTIVE); *count is a scratch counter that must be zero (the step
// launch before it clears counter word kListScratchWord).
cudaError_t launch_list_active(const Events& E, int* list, unsigned long long* count, cudaStream_t s);
cudaError_t launch_append_range(int* list, unsigned long long* count, int64_t base, int64_t n, cudaStream_t s);
cudaError_t launch_set_job(uint16_t* job_of, int64_t base, int64_t n, int job, cudaStream_t s);
// Persistent form; counters word 6 is the event cursor and must be zero.
cudaError_t launch_shower_persistent(const DevParams& P, const Events& E, const gaps_persistent_config& cfg,
                                     cudaStream_t s);
// Persistent form over a list, time-sliced: every event of list_in (length
// *n_in_dev when given, at most n_in) runs at most `cycles` (1..255) veto
// cycles; the still-active ones go to list_out through *out_count.  *cursor
// must be zero.
cudaError_t launch_shower_slice(const DevParams& P, const Events& E, const gaps_persistent_config& cfg,
                                const int* list_in, int64_t n_in, const unsigned long long* n_in_dev,
                                unsigned long long* cursor, int cycles, int* list_out, unsigned long long* out_count,
                                cudaStream_t s);
// The finalisation launchers visit positions 0 .. E.n - 1, mapped to events
// by R (the identity by default; E's per-event arrays are then indexed by
// the mapped event).
cudaError_t launch_validate(const DevParams& P, const Events& E, cudaStream_t s, const Ranges& R = Ranges{});
// buckets: int32 scratch [769] (counts, offsets, cursors); order: int32
// scratch [n_events].
cudaError_t launch_observables(const DevParams& P, const Events& E, int* buckets, int* order, cudaStream_t s,
                               const Ranges& R = Ranges{});
// Make CUDA load the observables' kernels on the current device now (it
// loads modules lazily by default, at their first use).
cudaError_t preload_observables();
// Histograms of the batch added to hist (doubles): one set for a single-job
// batch (scales from P, or from the device job-table entry *scale_src when
// given), one set per job for a multi-job batch (E.jobs and E.job_of set;
// the job count in counter word kJobCountWord).  Accumulated exactly in
// fixed point in the workspace's hist_fixed scratch, then converted.
cudaError_t launch_histograms(const DevParams& P, const DevParams* scale_src, const Events& E, double* hist,
                              cudaStream_t s);
// The exact fixed-point fills alone, added to acc (GAPS_HIST_FIXED_WORDS per
// set, not cleared).
cudaError_t launch_hist_fixed(const DevParams& P, const DevParams* scale_src, const Events& E, unsigned long long* acc,
                              cudaStream_t s, const Ranges& R = Ranges{});
// Sets 0 .. n_sets - 1 of acc added to hist as doubles (set j at hist + j *
// GAPS_HIST_DOUBLES; only sets with fills are touched).
cudaError_t launch_hist_finalize(const DevParams& P, const DevParams* scale_src, const DevParams* jobs, int n_sets,
                                 const unsigned long long* n_sets_dev, unsigned long long* acc, double* hist,
                                 cudaStream_t s);
cudaError_t launch_fill_job_of(uint16_t* job_of, const int64_t* begin, int n_jobs, int64_t n, cudaStream_t s);
cudaError_t launch_stats(const Events& E, gaps_stats* stats, cudaStream_t s);

}  // namespace gaps

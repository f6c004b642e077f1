// Batched launches of many small dense CP jobs (batch.cu), as the server uses them.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "../../include/ntf.h"

namespace ntf {
// ntf_batch_add with a caller-chosen id and submission time.
int batch_add(ntf_batch *b, const ntf_job *job, int64_t id, double t_submit);
// ntf_batch_tick.
int batch_tick(ntf_batch *b, int iters, int wait);
// Arena bytes the job would take (the admission test).
size_t batch_job_bytes(const ntf_batch *b, const ntf_job *job);
}  // namespace ntf

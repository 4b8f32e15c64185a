// Host worker threads shared by the library's host-side loops (host_pool.cu).
#pragma once
#include <functional>

namespace isg {

// Threads a host loop may use: min(16, hardware threads), at least 1.
int host_threads();

// Calls f(t) for t = 0 .. n-1, spread over the calling thread and up to
// host_threads() - 1 worker threads that live for the process, and returns
// when all calls have returned.  Calls from several threads are serialised;
// a call made from inside f runs inline; in a forked child the tasks run on
// fresh threads.  f must not throw.
void host_parallel(int n, const std::function<void(int)>& f);

}  // namespace isg

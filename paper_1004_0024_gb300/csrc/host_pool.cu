// Worker threads for the host-side loops of the library (CSR validation,
// slice extraction, threshold tables).  Creating a thread costs tens of
// microseconds, which made thread-per-call loops a visible part of creating
// and initialising a handle; these workers live for the process instead.
#include <unistd.h>

#include <algorithm>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "host_pool.h"

namespace isg {
namespace {

class Pool {
  public:
    explicit Pool(int workers) : pid_(getpid())
    {
        for (int w = 0; w < workers; ++w)
            th_.emplace_back([this, w] { loop(w + 1); });
    }
    int workers() const { return int(th_.size()); }
    pid_t pid() const { return pid_; }

    // f(id) on participants id = 0 .. n-1 (n <= workers + 1); the caller is
    // participant 0.  Returns when every participant has returned.
    void run(int n, const std::function<void(int)>& f)
    {
        {
            std::lock_guard<std::mutex> lk(m_);
            job_ = &f;
            n_ = n;
            pending_ = n - 1;
            ++gen_;
        }
        cv_.notify_all();
        f(0);
        std::unique_lock<std::mutex> lk(m_);
        done_.wait(lk, [this] { return pending_ == 0; });
        job_ = nullptr;
    }

  private:
    void loop(int id)
    {
        unsigned long long seen = 0;
        for (;;) {
            const std::function<void(int)>* job = nullptr;
            int n = 0;
            {
                std::unique_lock<std::mutex> lk(m_);
                cv_.wait(lk, [&] { return gen_ != seen; });
                seen = gen_;
                job = job_;
                n = n_;
            }
            // a worker outside this job's participants only records the
            // generation; a participant cannot miss its job, because run()
            // waits for it before the next generation starts
            if (job && id < n) {
                (*job)(id);
                std::lock_guard<std::mutex> lk(m_);
                if (--pending_ == 0)
                    done_.notify_one();
            }
        }
    }

    std::mutex m_;
    std::condition_variable cv_, done_;
    std::vector<std::thread> th_;
    const std::function<void(int)>* job_ = nullptr;
    int n_ = 0, pending_ = 0;
    unsigned long long gen_ = 0;
    pid_t pid_;
};

std::mutex g_pool_mu;          // one parallel loop at a time
thread_local bool g_in_task;   // a task that calls host_parallel runs it inline

Pool& pool()
{
    // never destroyed: the workers block on their condition variable until
    // the process exits
    static Pool* p = new Pool(host_threads() - 1);
    return *p;
}

}  // namespace

int host_threads()
{
    const unsigned hw = std::thread::hardware_concurrency();
    return int(std::max(1u, std::min(16u, hw)));
}

void host_parallel(int n, const std::function<void(int)>& f)
{
    if (n <= 0)
        return;
    if (n == 1 || g_in_task) {
        for (int t = 0; t < n; ++t)
            f(t);
        return;
    }
    // participants take tasks t = id, id + P, ... (P participants)
    auto strided = [&](int P) {
        return [&f, n, P](int id) {
            g_in_task = true;
            for (int t = id; t < n; t += P)
                f(t);
            g_in_task = false;
        };
    };
    std::lock_guard<std::mutex> lk(g_pool_mu);
    Pool& p = pool();
    if (p.pid() != getpid()) {
        // a forked child has none of the parent's workers: fresh threads
        const int P = std::min(n, host_threads());
        const std::function<void(int)> g = strided(P);
        std::vector<std::thread> th;
        for (int id = 1; id < P; ++id)
            th.emplace_back(g, id);
        g(0);
        for (auto& t : th)
            t.join();
        return;
    }
    const int P = std::min(n, p.workers() + 1);
    p.run(P, strided(P));
}

}  // namespace isg

// spill.cpp -- the spill file of the pinned host store and its IO thread.
#include "spill.h"

#include <unistd.h>

#include <chrono>
#include <cstdlib>
#include <string>
#include <vector>

#include "core.h"

namespace gbd {

SpillStore::~SpillStore() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        stop_ = true;
    }
    cv_.notify_all();
    if (th_.joinable()) th_.join();  // queued jobs finish first
    if (fd_ >= 0) close(fd_);
}

// One anonymous file per context: created in $TMPDIR (or /tmp) and unlinked
// at once, so it disappears with the process.
void SpillStore::open_file() {
    if (fd_ >= 0) return;
    const char* dir = std::getenv("TMPDIR");
    std::string path = std::string(dir && *dir ? dir : "/tmp") + "/gbd_spill_XXXXXX";
    std::vector<char> buf(path.begin(), path.end());
    buf.push_back('\0');
    fd_ = mkstemp(buf.data());
    GBD_REQUIRE(fd_ >= 0, GBD_ERR_HOST_OOM, "cannot create the spill file in " + path);
    unlink(buf.data());
    th_ = std::thread([this] { run(); });
}

long long SpillStore::region(long long prev_off, size_t prev_cap, size_t bytes, size_t* cap) {
    std::lock_guard<std::mutex> lk(mu_);
    if (prev_off >= 0 && prev_cap >= bytes) {
        *cap = prev_cap;
        return prev_off;
    }
    const long long off = end_;
    end_ += (long long)bytes;
    *cap = bytes;
    return off;
}

std::shared_ptr<SpillJob> SpillStore::submit(bool write, unsigned char* host, size_t bytes, long long off) {
    open_file();
    auto j = std::make_shared<SpillJob>();
    j->write = write;
    j->host = host;
    j->bytes = bytes;
    j->off = off;
    {
        std::lock_guard<std::mutex> lk(mu_);
        q_.push_back(j);
    }
    cv_.notify_one();
    return j;
}

int SpillStore::wait(const std::shared_ptr<SpillJob>& job, double timeout_ms) {
    const auto t0 = std::chrono::steady_clock::now();
    while (true) {
        const int s = job->state.load();
        if (s != 0) return s;
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms > timeout_ms) return 0;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

void SpillStore::run() {
    while (true) {
        std::shared_ptr<SpillJob> j;
        {
            std::unique_lock<std::mutex> lk(mu_);
            cv_.wait(lk, [&] { return stop_ || !q_.empty(); });
            if (q_.empty()) return;  // stop requested and nothing left
            j = q_.front();
            q_.pop_front();
        }
        size_t done = 0;
        bool ok = true;
        while (done < j->bytes) {
            const ssize_t r = j->write ? pwrite(fd_, j->host + done, j->bytes - done, j->off + (long long)done)
                                       : pread(fd_, j->host + done, j->bytes - done, j->off + (long long)done);
            if (r <= 0) { ok = false; break; }
            done += size_t(r);
        }
        j->state.store(ok ? 1 : -1);
    }
}

}  // namespace gbd

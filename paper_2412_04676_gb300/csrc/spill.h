// spill.h -- spill file of the pinned host store, with an IO thread.
//
// Sec. III.A / III.B.4 of arXiv:2412.04676: when the memory that holds saved
// environments is full, environments move to the next level of storage
// asynchronously through a load/save queue, and a task that needs one first
// waits until it is resident again ("fetching").  Here the pinned host store
// is bounded (gbd_config.host_store_bytes); environments the sweep does not
// need soon are written to one spill file by an IO thread and their pinned
// buffers freed; a spilled environment is read back into pinned memory by
// the same thread before it is unpacked.  Packages are self-contained
// (Sec. III.B.3), so a spilled stream is the packed stream, byte for byte.
#pragma once

#include <atomic>
#include <condition_variable>
#include <cstddef>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>

namespace gbd {

struct SpillJob {
    bool write = true;        // true: host memory -> file, false: file -> host memory
    unsigned char* host = nullptr;
    size_t bytes = 0;
    long long off = 0;        // file offset
    std::atomic<int> state{0};  // 0 queued or running, 1 done, -1 failed
};

class SpillStore {
  public:
    SpillStore() = default;
    ~SpillStore();
    SpillStore(const SpillStore&) = delete;
    SpillStore& operator=(const SpillStore&) = delete;

    // A file region for bytes: the id's previous region when it is large
    // enough, else a new one at the end of the file.
    long long region(long long prev_off, size_t prev_cap, size_t bytes, size_t* cap);
    std::shared_ptr<SpillJob> submit(bool write, unsigned char* host, size_t bytes, long long off);
    // Waits at most timeout_ms; returns the job state (0 if it is still running).
    static int wait(const std::shared_ptr<SpillJob>& job, double timeout_ms);

  private:
    void open_file();
    void run();
    int fd_ = -1;
    long long end_ = 0;
    std::mutex mu_;
    std::condition_variable cv_;
    std::deque<std::shared_ptr<SpillJob>> q_;
    bool stop_ = false;
    std::thread th_;
};

}  // namespace gbd

// apx_serve.h -- shared layout of the serving engine (host code in apx_api.cu,
// the persistent kernel in apx_serve.cu).
//
// The host appends requests to a ring in page-locked, device-mapped memory and
// publishes a running count of work items ("tickets"): a request's tickets are
// its template's preparation jobs (only when the template is not resident
// yet) followed by its overlap-save blocks.  Persistent CTAs claim tickets in
// order, never beyond the published count; a block waits (bounded) only for
// preparation jobs with smaller tickets, which CTAs that are already running
// hold.  The CTA that finishes a request's last item writes the request's
// status and then its sequence number to host-mapped completion words.
#pragma once

#include "apx_internal.cuh"

namespace apx {

constexpr int kServeThreads = 256;   // every persistent CTA (the FFT block body for W_block <= 8192)
constexpr int kServeWbMax = 8192;

// One request in flight (a ring slot, host-mapped; the host writes it before
// publishing its tickets and not again until the request is complete).
struct ServeSlot {
    Params p;           // the request; kernel-side pointers are its template's
    long long base;     // its first ticket
    int nprep;          // its preparation items (0 when the template is resident or being prepared)
    int njobs;          // preparation jobs of its template the blocks wait for
    int nitems;         // nprep + blocks
    unsigned seq;       // request number (never 0): written to the completion word
    int skip_prep;      // test hook: the preparation items are dropped
    int pad;
};

struct ServeHdr {       // host-mapped
    long long published;  // tickets published by the host
    int stop;             // the host asks the persistent CTAs to leave
    int pad;
};

struct ServeEnv {
    ServeHdr* hdr;            // host-mapped
    ServeSlot* slots;         // host-mapped ring
    int* tmap;                // host-mapped: slot of ticket t at tmap[t & tmask]
    long long tmask;
    unsigned long long* next; // device: the next ticket to claim
    int* done_items;          // device, per slot: items finished
    unsigned* dstatus;        // device, per slot: status bits (Params.status)
    unsigned* done_seq;       // host-mapped, per slot: sequence number once complete
    unsigned* fstatus;        // host-mapped, per slot: final status bits
    long long idle_cycles;    // a CTA leaves after this many SM cycles without work
};

cudaError_t launch_serve(const ServeEnv& env, int ctas, size_t smem, cudaStream_t st);
size_t serve_smem_bytes();

}  // namespace apx

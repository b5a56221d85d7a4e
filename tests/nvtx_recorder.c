/*
 * NVTX injection library used by the tracing tests (test infrastructure,
 * not part of the library).  A process started with NVTX_INJECTION64_PATH
 * naming this library hands it the NVTX core callbacks at its first NVTX
 * call; from then on every range push is recorded as "+<name>" and every
 * pop as "-", one per line, in call order.  nvtx_recorder_dump copies the
 * record out.
 */
#include <pthread.h>
#include <stdio.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

static pthread_mutex_t rec_mu = PTHREAD_MUTEX_INITIALIZER;
static char rec_buf[1 << 20];
static size_t rec_len;

static void rec_put(const char *s) {
    const size_t n = strlen(s);
    pthread_mutex_lock(&rec_mu);
    if (rec_len + n + 1 < sizeof rec_buf) {
        memcpy(rec_buf + rec_len, s, n);
        rec_len += n;
        rec_buf[rec_len++] = '\n';
    }
    pthread_mutex_unlock(&rec_mu);
}

static int rec_push(const char *name) {
    char line[512];
    snprintf(line, sizeof line, "+%s", name ? name : "");
    rec_put(line);
    return 0;
}

static int rec_pop(void) {
    rec_put("-");
    return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
    const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = NULL;
    unsigned int size = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) || !table ||
        size <= NVTX_CBID_CORE_RangePop)
        return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)rec_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)rec_pop;
    return 1;
}

/* Copies the record (NUL-terminated, truncated to cap - 1 bytes) and
 * returns its full length. */
size_t nvtx_recorder_dump(char *out, size_t cap) {
    pthread_mutex_lock(&rec_mu);
    const size_t n = rec_len < cap - 1 ? rec_len : cap - 1;
    memcpy(out, rec_buf, n);
    out[n] = 0;
    const size_t len = rec_len;
    pthread_mutex_unlock(&rec_mu);
    return len;
}

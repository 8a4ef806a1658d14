"""A randomised model of the fused BF16 encoder kernel's barrier protocol.

The kernel's roles (one thread issuing the x loads and the log-likelihood
MMAs, one issuing the statistics MMAs, six builder warps, eight softmax warps
per CTA, 1-4 CTAs per cluster) are modelled as generators that wait on
mbarrier phases and arrive on them exactly as the kernel does. Barriers follow
mbarrier semantics: an arrival count and a transaction-byte count per phase,
a parity wait that cannot tell phase n from phase n + 2. TMA copies, MMAs and
the cluster exchange's bulk copies complete asynchronously (queued, run in a
random order relative to the threads). A random scheduler interleaves
everything; the model checks that no buffer (landing buffer, Y stage, TMEM
log-likelihood buffer, gamma^T, statistics accumulator, exchange slot) is
overwritten while in use or read before it holds the right tile, and that the
run neither deadlocks nor loses a unit's statistics.

glo=True models FV_PREC_BF16X2: the posteriors' bf16 hi + lo pair of a tile
goes through the gamma^T buffer in two 64-row halves (lane quadrants 0-1,
then 2-3), each with its own full / free barrier, and the statistics
write-out's staging shares the buffer with the next unit's first half.

This is test infrastructure: nothing in the library imports it.
"""
import random

class Bar:
    def __init__(s, name, count):
        s.name, s.count, s.pending, s.phase, s.tx = name, count, count, 0, 0
    def arrive(s, n=1):
        s.pending -= n
        assert s.pending >= 0, s.name
        s._chk()
    def expect(s, n): s.tx += n
    def ctx(s, n):
        s.tx -= n
        s._chk()
    def _chk(s):
        if s.pending == 0 and s.tx == 0:
            s.phase += 1
            s.pending = s.count
    def ready(s, parity): return (s.phase & 1) != parity

class Fail(Exception): pass
def check(c, msg):
    if not c: raise Fail(msg)

def run(units_per_cluster, S, nstage, seed, drop=frozenset(), glo=False):
    rng = random.Random(seed)
    tiles = []
    for ui, n in enumerate(units_per_cluster):
        nt = (n + 127) // 128
        for t in range(nt):
            tiles.append((ui, t == 0, t == nt - 1))
    NT = len(tiles)
    lag = nstage - 1
    ctas = []
    for r in range(S):
        B = {}
        def mk(name, cnt): B[name] = Bar(name, cnt)
        mk('BFULL', 1); mk('XRFREE', 6)
        for s in range(2):
            mk(f'XRFULL{s}', 1); mk(f'AFULL{s}', 6); mk(f'STFREE{s}', 1); mk(f'LFULL{s}', 1)
            mk(f'LEMPTY{s}', 8); mk(f'XCHG{s}', 1)
        for q in range(4):
            mk(f'HXFULL{q}', 2); mk(f'HXFREE{q}', 2)   # two warps per quadrant (one arrival each here)
        mk('GFULL', 4 if glo else 8); mk('GFREE', 1); mk('SDONE', 1); mk('TEMPTY', 8)
        if glo:
            mk('GFULL2', 4); mk('GFREE2', 1)
        # gamma^T buffer as eight 4 KB units -> [tile, half, consumed]; stg: the write-out staging owner
        st = dict(ring=None, stage=[[None] * 6 for _ in range(2)], L=[None, None],
                  gbuf={k: None for k in range(8)}, stg={k: None for k in range(8)},
                  acc=None, xbuf=[[[None] * 4 for _ in range(S)] for _ in range(2)], hx=[[None, None] for _ in range(4)],
                  flushed=[])
        ctas.append(dict(B=B, st=st, mmaq=[], mmaq2=[], tmaq=[]))

    def build(c, i, part):
        B, st = c['B'], c['st']
        s = i % nstage
        j = i - nstage
        yield ('wait', B[f'XRFULL{i & 1}'], (i >> 1) & 1)
        check(st['ring'] == i, f'ring holds {st["ring"]} building {i}')
        yield ('step',)
        check(st['ring'] == i, f'ring changed while reading {i}')
        B['XRFREE'].arrive()          # registers hold the tile; the landing buffer may refill
        if j >= 0 and 'builder_stfree' not in drop:
            yield ('wait', B[f'STFREE{j & 1}'], (j >> 1) & 1)
        st['stage'][s][part] = i
        yield ('step',)
        B[f'AFULL{s}'].arrive()

    def builders(c, w):
        for i in range(NT):
            yield from build(c, i, w)

    def mma(c):
        # TMA loads + log-likelihood GEMMs (one thread)
        B, st = c['B'], c['st']
        q = c['mmaq']
        def load(i):
            b = B[f'XRFULL{i & 1}']
            b.expect(1); b.arrive()
            def land(i=i, b=b):
                check(st['ring_free'], f'landing buffer overwritten while in use ({i})')
                st['ring'] = i
                st['ring_free'] = False
                b.ctx(1)
            c['tmaq'].append(land)
        st['ring_free'] = True
        if NT > 0:
            load(0)
        yield ('wait', B['BFULL'], 0)
        for i in range(NT):
            s, b = i % nstage, i & 1
            if 'l_xrfree' not in drop:
                yield ('wait', B['XRFREE'], i & 1)
            st['ring_free'] = True
            if i + 1 < NT:
                load(i + 1)
            yield ('wait', B[f'AFULL{s}'], (i // nstage) & 1)
            if i >= 2 and 'l_lempty' not in drop:
                yield ('wait', B[f'LEMPTY{b}'], ((i >> 1) - 1) & 1)
            def lop(i=i, s=s, b=b):
                check(all(x == i for x in st['stage'][s]), f'L {i} stage {st["stage"][s]}')
                check(st['L'][b] is None or st['L'][b][1] == 'released', f'L buffer busy {st["L"][b]}')
                st['L'][b] = [i, 'L', 0]
            q.append(('op', lop))
            q.append(('commit', B[f'LFULL{b}']))
            yield ('step',)

    def smma(c):
        B, st = c['B'], c['st']
        q = c['mmaq2']
        for ns in range(NT):
            ui, first, last = tiles[ns]
            if first and ui > 0 and 'stats_tempty' not in drop:
                yield ('wait', B['TEMPTY'], (ui - 1) & 1)
            s = ns % nstage
            for half in ((0, 1) if glo else (0,)):
                full = 'GFULL2' if half else 'GFULL'
                yield ('wait', B[full], ns & 1)
                def op(ti=ns, s=s, ui=ui, first=first, half=half):
                    check(all(x == ti for x in st['stage'][s]), f'stats {ti} stage {st["stage"][s]}')
                    check(all(v is not None and v[0] == ti and v[1] == half for v in st['gbuf'].values()),
                          f'stats {ti}/{half} gamma {st["gbuf"]}')
                    check(all(o is None for o in st['stg'].values()), f'stats {ti} gamma under staging {st["stg"]}')
                    for v in st['gbuf'].values():
                        v[2] = True
                    if first and half == 0:
                        check(st['acc'] is None or st['acc'][2], f'acc overwritten before flush {st["acc"]}')
                        st['acc'] = [ui, 1, False]
                    else:
                        check(st['acc'][0] == ui, 'acc unit')
                q.append(('op', op))
                q.append(('commit', B['GFREE2' if half else 'GFREE']))
            q.append(('commit', B[f'STFREE{ns & 1}']))
            if last:
                def mark(ui=ui): st['acc_done'] = ui
                q.append(('op', mark))
                q.append(('commit', B['SDONE']))
            yield ('step',)

    def softmax(c, rank, h, q):
        B, st = c['B'], c['st']
        wid = h * 4 + q
        for i in range(NT):
            b = i & 1
            yield ('wait', B[f'LFULL{b}'], (i >> 1) & 1)
            check(st['L'][b] is not None and st['L'][b][0] == i and st['L'][b][1] != 'released', f'passA {i} {st["L"][b]}')
            yield ('step',)
            # pass A keeps the exponentials in registers: the TMEM buffer is released at once
            bl = B[f'LEMPTY{b}']
            if bl.pending == 1:
                st['L'][b][1] = 'released'
            bl.arrive()
            if i > 0 and 'softmax_hxfree' not in drop:
                yield ('wait', B[f'HXFREE{q}'], (i - 1) & 1)
            st['hx'][q][h] = i
            B[f'HXFULL{q}'].arrive()
            yield ('wait', B[f'HXFULL{q}'], i & 1)
            yield ('step',)
            check(st['hx'][q][0] == i and st['hx'][q][1] == i, f'hx {i} {st["hx"][q]}')
            B[f'HXFREE{q}'].arrive()
            if S > 1:
                j = i & 1
                if h == 0:
                    if q == 0:
                        B[f'XCHG{j}'].expect((S - 1) * 4); B[f'XCHG{j}'].arrive()
                    for pr in range(S):
                        if pr == rank: continue
                        peer = ctas[pr]
                        def land(peer=peer, i=i, j=j):
                            peer['st']['xbuf'][j][rank][q] = i
                            peer['B'][f'XCHG{j}'].ctx(1)
                        c['tmaq'].append(land)
                        yield ('step',)
                yield ('wait', B[f'XCHG{j}'], (i >> 1) & 1)
                yield ('step',)
                for pr in range(S):
                    if pr != rank:
                        check(st['xbuf'][j][pr][q] == i, f'xchg {i} from {pr} holds {st["xbuf"][j][pr]}')
                yield ('step',)
                for pr in range(S):
                    if pr != rank:
                        check(st['xbuf'][j][pr][q] == i, f'xchg {i} changed')
            ui, first, last = tiles[i]
            half = (q >> 1) if glo else 0
            # pass B writes: BF16 its 32 rows of component half h (unit 4h + q); BF16X2 its rows of the
            # 64-row half, hi at unit 2h + (q & 1) and lo at 4 + 2h + (q & 1); the staging uses unit 4h + q
            units = [2 * h + (q & 1), 4 + 2 * h + (q & 1)] if glo else [4 * h + q]
            slot = 4 * h + q
            if glo and half == 0 and first and ui > 0 and 'softmax_tempty' not in drop:
                yield ('wait', B['TEMPTY'], (ui - 1) & 1)   # the staging in this buffer is over
            if 'softmax_gfree' not in drop:
                if half == 0 and i >= 1:
                    yield ('wait', B['GFREE2' if glo else 'GFREE'], (i - 1) & 1)
                elif half == 1:
                    yield ('wait', B['GFREE'], i & 1)
            for u in units:
                check(st['stg'][u] is None, f'pass B {i} writes rows under staging {st["stg"]}')
                check(st['gbuf'][u] is None or st['gbuf'][u][2], f'pass B {i} overwrites unread gamma {st["gbuf"][u]}')
                st['gbuf'][u] = [i, half, False]
            yield ('step',)
            B['GFULL2' if half else 'GFULL'].arrive()
            if not last: continue
            yield ('wait', B['SDONE'], ui & 1)
            check(st.get('acc_done') == ui and st['acc'][0] == ui, f'flush {ui} acc {st["acc"]}')
            # the write-out stages through this warp's slot of the gamma^T buffer
            check(st['stg'][slot] is None and (st['gbuf'][slot] is None or st['gbuf'][slot][2]),
                  f'staging {ui} over unread gamma {st["gbuf"][slot]} / {st["stg"][slot]}')
            st['stg'][slot] = wid
            yield ('step',)
            check(st['acc'][0] == ui, 'acc changed during flush')
            check(st['stg'][slot] == wid, f'staging {ui} disturbed')
            st['stg'][slot] = None
            if B['TEMPTY'].pending == 1:
                st['acc'][2] = True
                st['flushed'].append(ui)
            B['TEMPTY'].arrive()

    gens = []
    for r, c in enumerate(ctas):
        c['B']['BFULL'].phase = 1
        gens.append(mma(c)); gens.append(smma(c))
        for w in range(6): gens.append(builders(c, w))
        for h in range(2):
            for q in range(4): gens.append(softmax(c, r, h, q))
    state = [None] * len(gens); done = [False] * len(gens)
    spin_rounds = 0
    while True:
        runnable = []
        spinners = []
        for k in range(len(gens)):
            if done[k]: continue
            op = state[k]
            if op is None or op[0] not in ('wait', 'spin') or (op[0] == 'wait' and op[1].ready(op[2])):
                runnable.append(('t', k))
            elif op[0] == 'spin':
                spinners.append(k)
        for r, c in enumerate(ctas):
            if c['tmaq']: runnable.append(('tma', r))
            if c['mmaq']: runnable.append(('mma', r))
            if c['mmaq2']: runnable.append(('mma2', r))
        if not runnable and spinners:
            # only pollers left: let one poll (if nothing changed it spins again -> deadlock check below)
            runnable = [('t', k) for k in spinners]
            spin_rounds += 1
            if spin_rounds > 50:
                raise Fail('deadlock: only pollers')
        else:
            spin_rounds = 0
        if not runnable:
            if all(done): break
            pend = [(k, state[k][1].name, state[k][2], state[k][1].phase) for k in range(len(gens)) if not done[k]]
            raise Fail(f'deadlock {pend[:6]}')
        kind, k = rng.choice(runnable)
        if kind == 'tma': ctas[k]['tmaq'].pop(0)()
        elif kind in ('mma', 'mma2'):
            op = ctas[k]['mmaq' if kind == 'mma' else 'mmaq2'].pop(0)
            if op[0] == 'op': op[1]()
            else: op[1].arrive()
        else:
            try: state[k] = next(gens[k])
            except StopIteration: done[k] = True
    for c in ctas:
        check(c['st']['flushed'] == list(range(len(units_per_cluster))), f'flushed {c["st"]["flushed"]}')


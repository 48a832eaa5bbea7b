"""The workspace layout of pcmm_cussen (plan, then one pass of strips),
mirrored from its documented structure so that GPU tests can read the plan
and the strip tables back (test infrastructure)."""
NLEV = 4
WAVE_ITEMS = 152 * 7 * 4     # one wave of the table kernel on a 152-SM GB300 (7 blocks per SM)
TARGET_WAVES = 4             # waves per pass, fewer when a pass exceeds 16 GiB
PASS_BYTES_CAP = 16 << 30


def _a256(x):
    return (x + 255) & ~255


def _level2_bound(w):
    lim, d = (1 << w) - 1, 0
    while (d + 1) * (d + 2) // 2 <= lim:
        d += 1
    return max(d, 1)


def layout(m, n, w, k, l=1):
    L = dict(m=m, n=n, w=w, k=k, l=l, nstrips=(n + k - 1) // k, n1max=min((1 << w) - 1, m))
    L["l2max"] = min(_level2_bound(w), L["n1max"])
    L["emax"] = min((1 << (w * k)) - 1, m)
    L["ptr_stride"] = L["n1max"] + (NLEV - 2) * L["l2max"]
    L["njb"] = (l + 31) // 32
    L["lp"] = L["njb"] * 32
    off = 256
    L["rank"] = off; off = _a256(off + L["nstrips"] * m * 2)
    L["nent"] = off; off = _a256(off + L["nstrips"] * 4)
    L["codes"] = off; off = _a256(off + L["nstrips"] * L["emax"] * 2)
    L["len"] = off; off = _a256(off + n * NLEV * 2)
    L["vN"] = off; off = _a256(off + n * L["l2max"] * 2)
    L["ptr"] = off; off = _a256(off + n * L["ptr_stride"] * 2)
    L["rank1"] = off; off = _a256(off + (n * 256 if k > 1 else 0))
    L["plan_bytes"] = off
    jac_ents = L["n1max"] + 2 * L["l2max"]
    aff_ents = L["l2max"] + (k * L["n1max"] + L["emax"] if k > 1 else 0)
    pref_ents = max(L["emax"], L["n1max"])
    L["item_u4"] = jac_ents * 6 * 32 + aff_ents * 4 * 32 + pref_ents * 2 * 32
    L["items_per_strip"] = 2 * L["njb"]
    return L


def single_pass_table(L):
    """Byte offset of the strip tables and their point count when one pass
    holds every strip and the gather does not split (m 2 njb >= 12288
    warps): the tables follow the plan and the pass's per-item scratch."""
    assert L["m"] * 2 * L["njb"] >= 12288, "the gather would split: partial sums precede the pass"
    ips = L["items_per_strip"]
    per_strip = ips * L["item_u4"] * 16 + _a256(L["emax"] * 2 * L["lp"] * 64)
    waves = TARGET_WAVES
    while waves > 1 and waves * WAVE_ITEMS // ips > PASS_BYTES_CAP // per_strip:
        waves -= 1
    S = max(1, min(L["nstrips"], waves * WAVE_ITEMS // ips))
    assert S == L["nstrips"], "more than one pass"
    table = L["plan_bytes"] + _a256(S * L["items_per_strip"] * L["item_u4"] * 16)
    return table, S * L["emax"] * 2 * L["lp"]

"""Naive list-of-agents predation (Section 5.1) used to pin the slab oracle.

Agents live in per-species dicts keyed by slot, the grass in a dict keyed by
(x, y); births take the smallest unused slot one at a time; conflicts are
settled by sorting each cell's claimants. None of the slab machinery
(compaction, ranked assignment, per-cell key tables) is used. Random draws are
the oracle's Philox (pinned separately against library implementations).
"""
from __future__ import annotations

import oracle

MOVES = {0: (-1, -1), 1: (0, -1), 2: (1, -1), 3: (-1, 0), 4: (1, 0), 5: (-1, 1), 6: (0, 1), 7: (1, 1)}


class BruteWorld:
    def __init__(self, side, seed, model, params, cap, n0, many_wolves=False, grass_off=False):
        self.L = side
        self.many_wolves = many_wolves
        self.grass_off = grass_off
        self.seed, self.model = seed, model
        self.p = [int(x) & 0xFFFFFFFF for x in params]
        self.gain = [self.p[0], self.p[1]]
        self.T = [self.p[2], self.p[3]]
        self.regrowth = self.p[4] if self.p[4] < 2**31 else self.p[4] - 2**32
        self.metab = [0 if grass_off else self.p[5], self.p[6]]
        self.cap = list(cap)
        self.t = 0
        self.next_id = list(n0)
        self.hw = list(n0)
        self.overflow = [0, 0]
        self.agents = [{}, {}]
        for s in range(2):
            for k in range(n0[s]):
                w = self.rand(0xFFFFFFFF, k, oracle.P_INIT_AGENT, s)
                cell = (w[0] * side * side) >> 32
                self.agents[s][k] = dict(x=cell % side, y=cell // side,
                                         e=(w[1] * 2 * self.gain[s]) >> 32, id=k, age=0)
        self.grass = {}
        for c in range(side * side):
            w = self.rand(0xFFFFFFFF, c, oracle.P_GRASS_INIT, 2)
            self.grass[(c % side, c // side)] = dict(
                grown=w[0] < self.p[7], countdown=(w[1] * max(self.regrowth, 0)) >> 32)

    def rand(self, step, slot, purpose, species):
        return [int(x) for x in oracle.philox([step, slot, purpose, species], [self.seed, self.model])]

    def draw(self, slot, purpose, species):
        return self.rand(self.t, slot, purpose, species)[0]

    def move(self, s):
        for slot in sorted(self.agents[s]):
            a = self.agents[s][slot]
            dx, dy = MOVES[self.draw(slot, oracle.P_MOVE, s) >> 29]
            a["x"] = (a["x"] + dx) % self.L
            a["y"] = (a["y"] + dy) % self.L
            a["e"] -= self.metab[s]
            a["age"] += 1

    def reproduce(self, s):
        parents = [slot for slot in sorted(self.agents[s])
                   if self.agents[s][slot]["e"] >= 0 and self.draw(slot, oracle.P_REPRO, s) < self.T[s]]
        births = 0
        for slot in parents:
            used = set(self.agents[s])
            free = [i for i in range(self.cap[s]) if i not in used]
            if not free:
                self.overflow[s] = 1
                break
            a = self.agents[s][slot]
            child_e = a["e"] // 2
            a["e"] -= child_e
            self.agents[s][free[0]] = dict(x=a["x"], y=a["y"], e=child_e,
                                           id=self.next_id[s] + births, age=0)
            births += 1
        self.next_id[s] += births
        self.hw[s] = max(self.hw[s], len(self.agents[s]))
        return len(parents), births

    def die(self, s):
        dead = [slot for slot, a in self.agents[s].items() if a["e"] < 0]
        for slot in dead:
            del self.agents[s][slot]
        return len(dead)

    def step(self):
        st = {}
        self.move(0)
        claims = {}
        for slot, a in self.agents[0].items():
            if self.grass[(a["x"], a["y"])]["grown"] and not self.grass_off:
                claims.setdefault((a["x"], a["y"]), []).append((self.draw(slot, oracle.P_PRIO, 0), slot))
        for cell, c in claims.items():
            winner = sorted(c)[0][1]
            self.agents[0][winner]["e"] += self.gain[0]
            self.grass[cell] = dict(grown=False, countdown=self.regrowth)
        st["grass_eaten"] = len(claims)
        st["parents0"], st["births0"] = self.reproduce(0)
        st["starved0"] = self.die(0)
        self.move(1)
        sheep_at = {}
        for slot, a in self.agents[0].items():
            sheep_at.setdefault((a["x"], a["y"]), []).append((self.draw(slot, oracle.P_VICTIM, 0), slot))
        wolf_claims = {}
        for slot, a in self.agents[1].items():
            cell = (a["x"], a["y"])
            if cell in sheep_at:
                wolf_claims.setdefault(cell, []).append((self.draw(slot, oracle.P_PRIO, 1), slot))
        eaten = 0
        for cell, c in wolf_claims.items():
            # one wolf per cell eats, or (variant) the k-th wolf the k-th sheep
            pairs = zip(sorted(c), sorted(sheep_at[cell])) if self.many_wolves else \
                [(sorted(c)[0], sorted(sheep_at[cell])[0])]
            for (_, wolf), (_, victim) in pairs:
                self.agents[1][wolf]["e"] += self.gain[1]
                del self.agents[0][victim]
                eaten += 1
        st["eaten"] = eaten
        st["parents1"], st["births1"] = self.reproduce(1)
        st["starved1"] = self.die(1)
        for g in self.grass.values():
            if not g["grown"]:
                g["countdown"] -= 1
                if g["countdown"] <= 0:
                    g["grown"] = True
        self.t += 1
        return st
